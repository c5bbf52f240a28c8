"""Tensor-core 16-point DFT stage (tcgen05.mma, bf16 operands, fp32 accumulate)
against numpy's FFT (a library routine independent of the CUDA path)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("batch", [1, 128, 1000, 4096])
@pytest.mark.parametrize("terms,tol", [(3, 3e-5), (1, 1e-2)])
def test_dft16_matches_numpy(batch, terms, tol):
    from paper_1411_0436_gb300 import vspec
    rng = np.random.default_rng(batch + terms)
    x = (rng.standard_normal((batch, 16)) + 1j * rng.standard_normal((batch, 16))) * 100.0
    x = x.astype(np.complex64)
    ref = np.fft.fft(x.astype(np.complex128), axis=1)
    dx = torch.from_numpy(x.view(np.float32).copy()).cuda()
    dy = torch.zeros_like(dx)
    vspec.vspec_tc_dft16(dx, dy, batch, terms)
    got = dy.cpu().numpy().view(np.complex64).astype(np.complex128).reshape(batch, 16)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"\nbatch {batch} terms {terms}: max error / max |Y| = {err:.3e}")
    assert err <= tol


def _dft16_inputs(batch):
    rng = np.random.default_rng(7)
    x = ((rng.standard_normal((batch, 16)) + 1j * rng.standard_normal((batch, 16))) * 100.0).astype(np.complex64)
    return x, np.fft.fft(x.astype(np.complex128), axis=1)


def test_wait_that_gives_up_reports_timeout_and_recovers():
    """A bounded wait limited to 0 polls gives up before the tensor cores
    finish: the call reports VSPEC_ERR_DEVICE_TIMEOUT (no fault, the context
    stays usable), and the next call with the default bound is correct."""
    from paper_1411_0436_gb300 import vspec
    batch = 512
    x, ref = _dft16_inputs(batch)
    dx = torch.from_numpy(x.view(np.float32).copy()).cuda()
    dy = torch.zeros_like(dx)
    try:
        vspec.vspec_set_wait_limit(0)
        with pytest.raises(vspec.VspecError) as e:
            vspec.vspec_tc_dft16(dx, dy, batch, 3)
        assert e.value.status == vspec.ERR_DEVICE_TIMEOUT
    finally:
        vspec.vspec_set_wait_limit(-1)
    vspec.vspec_tc_dft16(dx, dy, batch, 3)
    got = dy.cpu().numpy().view(np.complex64).astype(np.complex128).reshape(batch, 16)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 3e-5


def test_tensor_plan_timeout_flag_is_reported_and_cleared(oracle_mod):
    """The tensor-core row kernel under a 0-poll wait raises the plan's flag:
    vspec_plan_check reports it once and clears it; the plan then runs
    normally and matches the oracle."""
    from parity_util import ATOL_TC, assert_close
    from paper_1411_0436_gb300 import vspec, workloads
    bank = workloads.Bank(32768, 8, 2, workloads.PFB, workloads.WIN_HANN, 6, rho=0.3)
    x = workloads.generate(bank, 77)
    d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
    with vspec.Plan(bank.nchan, bank.ntaps, 2, bank.mode, bank.window, vspec.PLAN_TENSOR) as plan:
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        try:
            vspec.vspec_set_wait_limit(0)
            plan.execute(d_in, bank.nspectra, acc)
            torch.cuda.synchronize()
        finally:
            vspec.vspec_set_wait_limit(-1)
        with pytest.raises(vspec.VspecError) as e:
            plan.check()
        assert e.value.status == vspec.ERR_DEVICE_TIMEOUT
        plan.check()  # cleared
        plan.dump(acc)
        plan.execute(d_in, bank.nspectra, acc)
        torch.cuda.synchronize()
        plan.check()
        got = acc.cpu().numpy().astype(np.float64).reshape(-1, 4)
    o = oracle_mod.channelize(x, bank.nchan, bank.ntaps, 2, bank.nspectra, bank.mode, bank.window)
    assert_close(got, o, atol=ATOL_TC, what="tensor plan after a timeout")


def test_injected_timeout_is_reported_once():
    """Host-side injection of the timeout flag: reported by the next check,
    then cleared; plans without device-side waits refuse the injection."""
    from paper_1411_0436_gb300 import vspec
    with vspec.Plan(4096, 8, 2, vspec.PFB, vspec.WIN_HANN, vspec.PLAN_TENSOR) as plan:
        plan.check()
        plan.inject_timeout()
        with pytest.raises(vspec.VspecError) as e:
            plan.check()
        assert e.value.status == vspec.ERR_DEVICE_TIMEOUT
        plan.check()
    with vspec.Plan(4096, 8, 2, vspec.PFB, vspec.WIN_HANN) as plan:
        plan.check()  # no flag to report
        with pytest.raises(vspec.VspecError) as e:
            plan.inject_timeout()
        assert e.value.status == vspec.ERR_UNSUPPORTED
