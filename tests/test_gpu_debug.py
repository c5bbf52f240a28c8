"""The bounds-checked debug build (libvspec_debug.so, -DVSPEC_DEBUG).

Its kernels check every chunk-scratch, partial-sum slot, tile and input-frame
index against the buffers the plan and the call own, record a failed check in
a device status word and skip the access instead of trapping. These tests run
the small parity shapes (one per kernel form) through that build in a child
process (VSPEC_LIBRARY=debug), compare each result with the FP64 oracle and
require the status word to stay clear; on the release build the status call
is refused without touching the GPU.
"""
import ctypes
import json
import os
import subprocess
import sys

import pytest

from paper_1411_0436_gb300 import build as vbuild
from paper_1411_0436_gb300 import vspec

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
import numpy as np
import torch
sys.path.insert(0, os.environ["VSPEC_ROOT"]); sys.path.insert(0, os.path.join(os.environ["VSPEC_ROOT"], "tests"))
import oracle
from parity_util import metrics
from paper_1411_0436_gb300 import vspec, workloads
from paper_1411_0436_gb300.workloads import DIRECT, PFB, WIN_HANN, WIN_RECT, Bank, Tone
lib = vspec.load()
assert lib._name.endswith("libvspec_debug.so"), lib._name
vspec.vspec_debug_flags(clear=True)
# (nchan, taps, npol, mode, window, spectra, flags): register-column kernel A
# for 2..64-point columns, direct-mode columns, the tap-gather form, the
# general kernel A (single-pol), one-row transforms with the FIR in kernel B,
# the general row kernel, compensated plans, several chunks, the persistent ring form
shapes = [(4096, 8, 2, PFB, WIN_HANN, 19, 0), (32768, 8, 2, PFB, WIN_HANN, 67, 1),
          (131072, 8, 2, PFB, WIN_HANN, 5, 0), (524288, 1, 2, DIRECT, WIN_RECT, 3, 0),
          (1 << 19, 8, 2, PFB, WIN_HANN, 3, 0), (1024, 8, 1, PFB, WIN_HANN, 64, 0),
          (8192, 2, 1, PFB, WIN_HANN, 7, 0), (65536, 4, 1, PFB, WIN_HANN, 6, 0),
          (2048, 5, 2, PFB, WIN_RECT, 40, 4), (16384, 1, 2, DIRECT, WIN_HANN, 9, 4),
          (131072, 8, 2, PFB, WIN_HANN, 37, 16), (32768, 8, 2, PFB, WIN_HANN, 131, 16)]
out = []
for n, p, npol, mode, win, s, flags in shapes:
    bank = Bank(n, p, npol, mode, win, s, rho=0.3 if npol == 2 else 0.0, tones=(Tone(30.0, n * 0.3 + 0.4, (0,)),))
    x = workloads.generate(bank, 900 + n)
    with vspec.Plan(n, p, npol, mode, win, flags) as plan:
        if n == 32768 and flags & 16:
            plan.set_ring(slot_spectra=4, ring_slots=2, lookahead=1)  # many slots through a small ring
        elif n == 32768:
            plan.tune(chunk_spectra=16)  # several chunks
        d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        plan.execute(d_in, s, acc)
        torch.cuda.synchronize()
        g = acc.cpu().numpy().astype(np.float64)
        desc = plan.describe()
    o = oracle.channelize(x, n, p, npol, s, mode, win)
    m = metrics(g.reshape(n, 4) if npol == 2 else g, o)
    out.append({"shape": [n, p, npol, mode, win, s, flags], "plan": desc, "ratio": m["ratio"]})
print(json.dumps({"flags": vspec.vspec_debug_flags(clear=True), "cases": out}))
"""


def test_release_build_refuses_debug_status():
    lib = vspec.load()
    w = ctypes.c_uint(7)
    assert lib.vspec_debug_flags(ctypes.byref(w), 0) == vspec.ERR_UNSUPPORTED


def test_debug_build_exports_every_declared_symbol():
    vbuild.build()
    lib = ctypes.CDLL(vbuild.LIB_DEBUG)
    for name in vspec.declared_functions():
        assert hasattr(lib, name), f"{name} missing from the debug build"


@pytest.mark.gpu
def test_debug_build_parity_and_clean_status():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    vbuild.build()
    env = dict(os.environ, VSPEC_LIBRARY="debug", VSPEC_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for case in res["cases"]:
        print(f"\n{case['shape']} {case['plan']}: tolerance use {case['ratio']:.3f}")
        assert case["ratio"] <= 1.0, case
    assert res["flags"] == 0, f"bounds checks fired: {res['flags']:#x}"
