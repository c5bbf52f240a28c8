"""Full-size workloads: every bank of the five workload configurations, GPU vs
the FP64 oracle over all channels, in the launch configuration the benchmark
uses (one plan, one vspec_execute over all spectra of the dump)."""
import time

import numpy as np
import pytest

from parity_util import assert_close
from paper_1411_0436_gb300 import workloads
from test_gpu_parity import run_gpu, run_oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CASES = [(name, i) for name in ("c1", "c2", "c3", "c4", "c5")
         for i in range(len(workloads.CONFIGS[name]))]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name,idx", CASES, ids=[f"{n}_bank{i}" for n, i in CASES])
def test_workload_matches_oracle(oracle_mod, name, idx):
    bank = workloads.CONFIGS[name][idx]
    x = workloads.generate(bank, workloads.config_seed(name, idx))
    t0 = time.time()
    g = run_gpu(bank, x)
    t1 = time.time()
    o = run_oracle(oracle_mod, bank, x)
    t2 = time.time()
    m = assert_close(g, o, what=f"{name}[{idx}]")
    print(f"\n{name}[{idx}] N={bank.nchan} S={bank.nspectra}: normalised max err {m['pure']:.3e}, "
          f"tolerance use {m['ratio']:.3f}, gpu {t1 - t0:.2f}s oracle {t2 - t1:.1f}s")


@pytest.mark.parametrize("name", ["c2", "c4"])
def test_workload_tensor_core_path(oracle_mod, name):
    """The tensor-core form on the benchmark and precision-stress workloads:
    within the tensor-core tolerance; the error is printed beside the FP32
    path's."""
    from parity_util import ATOL_TC, metrics
    from paper_1411_0436_gb300.vspec import PLAN_TENSOR
    bank = workloads.CONFIGS[name][0]
    x = workloads.generate(bank, workloads.config_seed(name))
    o = run_oracle(oracle_mod, bank, x)
    g = run_gpu(bank, x, flags=PLAN_TENSOR)
    m = assert_close(g, o, atol=ATOL_TC, what=f"{name} tensor")
    f = metrics(run_gpu(bank, x), o)
    from paper_1411_0436_gb300.vspec import PLAN_KAHAN
    k = assert_close(run_gpu(bank, x, flags=PLAN_KAHAN), o, what=f"{name} kahan")
    tk = assert_close(run_gpu(bank, x, flags=PLAN_KAHAN | PLAN_TENSOR), o, atol=ATOL_TC,
                      what=f"{name} tensor+kahan")
    print(f"\n{name}: normalised max error: fp32 {f['pure']:.3e}, fp32+kahan {k['pure']:.3e}, "
          f"tensor {m['pure']:.3e}, tensor+kahan {tk['pure']:.3e}")
