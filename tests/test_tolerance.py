"""Pins of the FP32 parity tolerance itself (tests/parity_util.py).

The per-channel relative term r(N) = (log2(N)/4 + 2) u is derived from the
FP32 rounding of a correct implementation. These tests check it against
implementations outside the CUDA path:

  * a single-precision FFT with correctly rounded twiddles (scipy.fft on
    complex64) over the FP32 pre-filter output, summed exactly, must pass:
    the tolerance admits a correct FP32 channelizer;
  * the FP64 oracle's own result rounded to FP32 must pass with room;
  * the same channelizer with its pre-filter output rounded to FP16 (a
    half-precision stage, 2^-11 relative error per sample) must fail, and so
    must plain FP32 summation over a long dump: the tolerance catches what it
    is meant to catch.

Workloads: the 32768- and 131072-channel dual-pol PFB recipes (two tones;
the 40 dB tone), shortened to a few dozen spectra so the CPU suite stays fast.
"""
import numpy as np
import pytest

from parity_util import metrics, rtol_fp32
from paper_1411_0436_gb300 import workloads

sfft = pytest.importorskip("scipy.fft")


def _single_precision_channelizer(x, bank, h, half_stage=False, f32_sum=False):
    """Accumulated XX, YY, Re XY*, Im XY* from an FP32 FIR and scipy's FP32 FFT."""
    N, P, S = bank.nchan, bank.taps_used, bank.nspectra
    xf = (x[..., 0].astype(np.float32) + 1j * x[..., 1].astype(np.float32)).astype(np.complex64)
    acc = np.zeros((N, 4), np.float32 if f32_sum else np.float64)
    for s in range(S):
        fr = xf[s * N:(s + P) * N].reshape(P, N, 2)
        y = np.einsum("tn,tnp->np", h, fr).astype(np.complex64)
        if half_stage:
            y = (y.real.astype(np.float16).astype(np.float32)
                 + 1j * y.imag.astype(np.float16).astype(np.float32)).astype(np.complex64)
        Y = sfft.fft(y, axis=0)
        X0, X1 = Y[:, 0], Y[:, 1]
        d = np.stack([X0.real * X0.real + X0.imag * X0.imag, X1.real * X1.real + X1.imag * X1.imag,
                      X0.real * X1.real + X0.imag * X1.imag, X0.imag * X1.real - X0.real * X1.imag], 1)
        acc += d.astype(acc.dtype)
    return acc.astype(np.float64)


@pytest.mark.parametrize("name,spectra", [("c2", 48), ("c4", 24)])
def test_tolerance_admits_fp32_and_rejects_half_precision(oracle_mod, name, spectra):
    bank = workloads.config_banks(name)[0].with_spectra(spectra)
    x = workloads.generate(bank, workloads.config_seed(name))
    o = oracle_mod.channelize(x, bank.nchan, bank.ntaps, bank.npol, bank.nspectra, bank.mode, bank.window)
    h = oracle_mod.coeffs(bank.nchan, bank.ntaps, bank.mode, bank.window).astype(np.float32)
    h = h.reshape(bank.taps_used, bank.nchan)
    good = metrics(_single_precision_channelizer(x, bank, h), o)
    assert good["ratio"] <= 1.0, good
    rounded = metrics(o.astype(np.float32).astype(np.float64), o)
    assert rounded["ratio"] <= 0.5, rounded
    half = metrics(_single_precision_channelizer(x, bank, h, half_stage=True), o)
    assert half["ratio"] > 2.0, half
    print(f"\n{name}: r(N) = {rtol_fp32(bank.nchan) / 2.0 ** -24:.2f} u; tolerance use: FP32 FFT "
          f"{good['ratio']:.2f}, oracle rounded to FP32 {rounded['ratio']:.2f}, FP16 stage {half['ratio']:.1f}")


def test_tolerance_rejects_long_plain_fp32_sums(oracle_mod):
    """Plain FP32 summation of many spectra of a strong tone drifts beyond
    r(N): the tolerance forces compensated or split sums on long dumps."""
    N = 1 << 12  # the same recipe on a shorter transform, so that 1024 spectra stay fast
    bank = workloads.Bank(N, 8, 2, workloads.PFB, workloads.WIN_HANN, 1024, sigma=4.0,
                          tones=(workloads.Tone(40.0, 0.2 * N, (0, 1)),))
    x = workloads.generate(bank, 5)
    o = oracle_mod.channelize(x, N, 8, 2, bank.nspectra, bank.mode, bank.window)
    h = oracle_mod.coeffs(N, 8, bank.mode, bank.window).astype(np.float32).reshape(8, N)
    exact = metrics(_single_precision_channelizer(x, bank, h), o)
    plain = metrics(_single_precision_channelizer(x, bank, h, f32_sum=True), o)
    assert exact["ratio"] <= 1.0, exact
    assert plain["ratio"] > 1.0, plain
