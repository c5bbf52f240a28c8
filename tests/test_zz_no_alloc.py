"""The allocation-free entry point against the plan-based path.

vspec_execute_noalloc serves callers that cannot call cudaMalloc: an
application that owns all device memory through its own pool, or a real-time
capture loop where an allocation (which can synchronise the device) would
stall the data path and drop samples. It keeps all of its working memory in a
fixed array inside the library, and must give what vspec_execute gives (and
what the FP64 oracle gives) within the FP32 tolerance.
This file is collected last so that a run stopping at the first failure has
run every other test first.
"""
import numpy as np
import pytest

from parity_util import assert_close
from paper_1411_0436_gb300 import workloads
from paper_1411_0436_gb300.workloads import DIRECT, PFB, WIN_HANN, WIN_RECT, Bank, Tone

torch = pytest.importorskip("torch")


def _plan_path(bank: Bank, d_in) -> np.ndarray:
    from paper_1411_0436_gb300.vspec import Plan
    with Plan(bank.nchan, bank.ntaps, bank.npol, bank.mode, bank.window) as plan:
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        plan.execute(d_in, bank.nspectra, acc)
        torch.cuda.synchronize()
        return acc.cpu().numpy().astype(np.float64)


@pytest.mark.gpu
def test_noalloc_matches_plan_path_on_consecutive_calls(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_0436_gb300 import vspec
    banks = [
        Bank(32768, 8, 2, PFB, WIN_HANN, 37, rho=0.3, tones=(Tone(30.0, 3277.05, (0, 1)),)),
        Bank(4096, 1, 1, DIRECT, WIN_RECT, 11, tones=(Tone(25.0, 100.5, (0,)),)),
        # one-row transforms (no column pass), the smallest size, taps that
        # leave leading zero slots in the FIR window, windowed direct mode
        Bank(1024, 8, 1, PFB, WIN_HANN, 64, tones=(Tone(30.0, 123.4, (0,)),)),
        Bank(16, 8, 2, PFB, WIN_HANN, 9, rho=0.3),
        Bank(8192, 3, 2, PFB, WIN_HANN, 21, rho=0.3, tones=(Tone(20.0, 1000.25, (0, 1)),)),
        Bank(16384, 5, 2, PFB, WIN_RECT, 13),
        Bank(2048, 1, 2, DIRECT, WIN_HANN, 40, rho=0.3),
    ]
    for call, bank in enumerate(banks):  # calls in a row; each one rebuilds the tables
        x = workloads.generate(bank, 4242 + call)
        d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
        ref = _plan_path(bank, d_in)
        acc = torch.zeros(ref.size, dtype=torch.float32, device="cuda")
        vspec.vspec_execute_noalloc(d_in, bank.nchan, bank.ntaps, bank.npol, bank.mode, bank.window,
                                    bank.nspectra, acc)
        torch.cuda.synchronize()
        got = acc.cpu().numpy().astype(np.float64)
        shape = (bank.nchan, 4) if bank.npol == 2 else (bank.nchan,)
        assert_close(got.reshape(shape), ref.reshape(shape), what=f"noalloc call {call} vs plan")
        o = oracle_mod.channelize(x, bank.nchan, bank.ntaps, bank.npol, bank.nspectra, bank.mode,
                                  bank.window)
        assert_close(got.reshape(shape), o, what=f"noalloc call {call} vs oracle")
    # the same problem twice more: the tables are reused, the partial sums cleared
    bank = banks[-1]
    x = workloads.generate(bank, 4242 + len(banks) - 1)
    d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
    acc = torch.zeros(bank.nchan * 4, dtype=torch.float32, device="cuda")
    for _ in range(2):
        vspec.vspec_execute_noalloc(d_in, bank.nchan, bank.ntaps, bank.npol, bank.mode, bank.window,
                                    bank.nspectra, acc)
    torch.cuda.synchronize()
    o = oracle_mod.channelize(x, bank.nchan, bank.ntaps, bank.npol, bank.nspectra, bank.mode, bank.window)
    assert_close(acc.cpu().numpy().astype(np.float64).reshape(bank.nchan, 4), 2 * o, what="noalloc repeated")

    # beyond the fixed scratch: rejected with a clear reason, nothing launched
    lib = vspec.load()
    acc = torch.zeros(65536 * 4, dtype=torch.float32, device="cuda")
    d_in = torch.zeros(65536 * 4 * 8, dtype=torch.uint8, device="cuda")
    st = lib.vspec_execute_noalloc(d_in.data_ptr(), 65536, 8, 2, PFB, WIN_HANN, 1, acc.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert st == vspec.ERR_UNSUPPORTED
    assert "32768" in lib.vspec_last_error().decode()
