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
