"""Batches in persistent mode: every bank's work as tickets of one cooperative
launch (kernel-A tiles, then rows, then folds), against the FP64 oracle.

Covers every ticket body (register-column kernel A for PFB and direct mode,
the 2048-point row kernel, the one-row transforms of 2048 and of up to 1024
channels), banks with no spectra, ragged spectrum counts, the full c5
workload, bitwise reproducibility, switching back to per-bank kernels, the
refusal of banks the kernel has no body for, and a wait that gives up
(injected from the host by a done counter that starts one short: no GPU
fault is involved).
"""
import numpy as np
import pytest

from parity_util import assert_close
from paper_1411_0436_gb300 import workloads
from paper_1411_0436_gb300.workloads import DIRECT, PFB, WIN_HAMMING, WIN_HANN, WIN_RECT, Bank, Tone
from test_gpu_parity import run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def tone_bank(n, p, mode, win, s):
    return Bank(n, p, 2, mode, win, s, rho=0.3, tones=(Tone(25.0, n * 0.23 + 0.4, (0,)),))


MIXED = [tone_bank(1024, 8, PFB, WIN_HANN, 41), tone_bank(4096, 1, DIRECT, WIN_RECT, 19),
         tone_bank(16384, 8, PFB, WIN_HANN, 70), tone_bank(32768, 5, PFB, WIN_HAMMING, 9),
         tone_bank(65536, 1, DIRECT, WIN_HANN, 33), tone_bank(2048, 8, PFB, WIN_HANN, 37),
         tone_bank(512, 3, PFB, WIN_HANN, 5), tone_bank(131072, 8, PFB, WIN_HANN, 0),
         tone_bank(262144, 8, PFB, WIN_HANN, 3), tone_bank(16, 8, PFB, WIN_HANN, 9)]


def run_batch(banks, xs, persistent=True, repeat=1, autotune=False):
    from paper_1411_0436_gb300.vspec import Batch
    with Batch([(b.nchan, b.ntaps, b.npol, b.mode, b.window) for b in banks]) as batch:
        d_in = [torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda() for x in xs]
        accs = [torch.zeros(batch.out_floats(i), dtype=torch.float32, device="cuda") for i in range(len(banks))]
        ns = [b.nspectra for b in banks]
        if autotune:
            batch.autotune(d_in, ns, accs, reps=1)
        if persistent:
            batch.set_persistent(True)
            assert batch.persistent
        for _ in range(repeat):
            batch.execute(d_in, ns, accs)
        torch.cuda.synchronize()
        batch.check()
        return [a.cpu().numpy().astype(np.float64).reshape(b.nchan, 4) for a, b in zip(accs, banks)]


def test_persistent_mixed_banks_match_oracle(oracle_mod):
    xs = [workloads.generate(b, 800 + i) for i, b in enumerate(MIXED)]
    got = run_batch(MIXED, xs)
    for b, g, x in zip(MIXED, got, xs):
        if b.nspectra == 0:
            assert not np.any(g), "a bank without spectra must leave its accumulator alone"
            continue
        m = assert_close(g, run_oracle(oracle_mod, b, x), what=f"persistent bank {b.nchan}")
        print(f"\nbank {b.nchan} x {b.nspectra}: max err / RMS {m['pure']:.2e}, tolerance use {m['ratio']:.3f}")


def test_persistent_is_reproducible_and_accumulates(oracle_mod):
    banks = MIXED[:6]
    xs = [workloads.generate(b, 900 + i) for i, b in enumerate(banks)]
    a = run_batch(banks, xs, repeat=2)
    b2 = run_batch(banks, xs, repeat=2)
    for i, (u, v) in enumerate(zip(a, b2)):
        assert np.array_equal(u, v), f"bank {i} differs between identical runs"
    for b, g, x in zip(banks, a, xs):
        assert_close(g, 2.0 * run_oracle(oracle_mod, b, x), what=f"persistent bank {b.nchan}, two calls")


def test_persistent_after_autotune_and_back(oracle_mod):
    """Autotuned plans (trimmed chunks), the persistent launch, then per-bank kernels again."""
    from paper_1411_0436_gb300.vspec import Batch
    banks = [MIXED[1], MIXED[2], MIXED[4], MIXED[5]]
    xs = [workloads.generate(b, 950 + i) for i, b in enumerate(banks)]
    refs = [run_oracle(oracle_mod, b, x) for b, x in zip(banks, xs)]
    with Batch([(b.nchan, b.ntaps, b.npol, b.mode, b.window) for b in banks]) as batch:
        d_in = [torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda() for x in xs]
        accs = [torch.zeros(batch.out_floats(i), dtype=torch.float32, device="cuda") for i in range(len(banks))]
        ns = [b.nspectra for b in banks]
        batch.autotune(d_in, ns, accs, reps=1)
        for persistent in (True, False, True):
            batch.set_persistent(persistent)
            for a in accs:
                a.zero_()
            batch.execute(d_in, ns, accs)
            torch.cuda.synchronize()
            batch.check()
            for b, a, o in zip(banks, accs, refs):
                assert_close(a.cpu().numpy().astype(np.float64).reshape(o.shape), o,
                             what=f"bank {b.nchan} persistent={persistent}")


def test_persistent_refuses_banks_without_a_body():
    from paper_1411_0436_gb300.vspec import ERR_UNSUPPORTED, Batch, VspecError
    for bank in ((1 << 20, 8, 2, PFB, WIN_HANN), (8192, 8, 1, PFB, WIN_HANN), (32768, 4, 2, PFB, WIN_HANN)):
        with Batch([(4096, 8, 2, PFB, WIN_HANN), bank]) as batch:
            with pytest.raises(VspecError) as e:
                batch.set_persistent(True)
            assert e.value.status == ERR_UNSUPPORTED, bank
    with Batch([(4096, 8, 2, PFB, WIN_HANN)] * 17) as batch:
        with pytest.raises(VspecError) as e:
            batch.set_persistent(True)
        assert e.value.status == ERR_UNSUPPORTED


def test_persistent_wait_that_gives_up_is_reported_and_recovers(oracle_mod):
    from paper_1411_0436_gb300.vspec import ERR_DEVICE_TIMEOUT, Batch, VspecError, vspec_set_wait_limit
    banks = [MIXED[2], MIXED[4]]
    xs = [workloads.generate(b, 970 + i) for i, b in enumerate(banks)]
    refs = [run_oracle(oracle_mod, b, x) for b, x in zip(banks, xs)]
    with Batch([(b.nchan, b.ntaps, b.npol, b.mode, b.window) for b in banks]) as batch:
        d_in = [torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda() for x in xs]
        accs = [torch.zeros(batch.out_floats(i), dtype=torch.float32, device="cuda") for i in range(len(banks))]
        ns = [b.nspectra for b in banks]
        batch.set_persistent(True)
        vspec_set_wait_limit(20000)  # about 2 ms per wait
        try:
            batch.inject_stall(1)
            batch.execute(d_in, ns, accs)
            torch.cuda.synchronize()
            with pytest.raises(VspecError) as e:
                batch.check()
            assert e.value.status == ERR_DEVICE_TIMEOUT
            batch.check()  # reported once
        finally:
            vspec_set_wait_limit(-1)
        for a in accs:
            a.zero_()
        batch.execute(d_in, ns, accs)
        torch.cuda.synchronize()
        batch.check()
        for b, a, o in zip(banks, accs, refs):
            assert_close(a.cpu().numpy().astype(np.float64).reshape(o.shape), o, what=f"bank {b.nchan} after a timeout")


@pytest.mark.slow
def test_persistent_c5_workload(oracle_mod):
    banks = workloads.CONFIGS["c5"]
    xs = [workloads.generate(b, workloads.config_seed("c5", i)) for i, b in enumerate(banks)]
    got = run_batch(banks, xs)
    for b, g, x in zip(banks, got, xs):
        m = assert_close(g, run_oracle(oracle_mod, b, x), what=f"c5 persistent bank {b.nchan}")
        print(f"\nc5 bank {b.nchan} x {b.nspectra}: max err / RMS {m['pure']:.2e}, tolerance use {m['ratio']:.3f}")
