"""Comparison of the CUDA path's accumulated spectra with the FP64 oracle.

Tolerance, per channel k after S spectra of an N-channel transform:

  auto terms XX, YY:   |G_k - O_k| <= ATOL * RMS(O) + r(N) * |O_k|
  cross terms Re, Im:  |G_k - O_k| <= ATOL * sqrt(RMS(XX) RMS(YY))
                                      + r(N) * sqrt(XX_k YY_k)

  r(N) = (C_FFT * log2 N + C_OUT) * u,   u = 2^-24 (FP32 unit roundoff),
  C_FFT = 1/4, C_OUT = 2.

ATOL = 1e-5 is the error normalised to the spectrum RMS that the FP32 path
must meet. It binds every channel whose power is within a hundred or so of
the RMS. It cannot bind a channel far above the RMS (a tone), because the
FP32 format itself cannot: a channel at T times the RMS, stored in FP32, is
off by up to T * u / 2 of its value, which passes 1e-5 of the RMS once T
exceeds about 170 (the precision-stress workload's tone sits at 361 times
the RMS). For such channels the bound is relative, r(N) * |O_k|, built from
the two sources of FP32 error:

  * The transform. Each of the log2 N radix-2 levels of the DFT (however the
    levels are grouped into radix-8/16 passes) rounds the values on the
    tone's path once or twice. The rounding errors of the many values that
    feed a channel largely cancel, but those of the last levels, where the
    tone's energy sits in few values, do not, and they repeat from spectrum
    to spectrum as the tone repeats. A single-precision FFT with correctly
    rounded twiddles (scipy.fft on complex64, summed in FP64) shows
    0.10-0.12 u per level in power on these workloads; C_FFT = 1/4 per level
    allows twice that. tests/test_tolerance.py checks that such an FFT
    passes and that a transform carrying 2^-14 relative noise fails.
  * Detection, summation and output: |X|^2 rounds once (up to u), the sum
    over spectra adds at most about u when it is compensated or split into
    short runs (the kernels' two-level and Kahan sums), and the stored FP32
    result rounds by u/2. C_OUT = 2 covers the three.

The pure normalised error max_k |G - O| / RMS is reported alongside.

The tensor-core path must meet ATOL_TC = 1e-3 of the RMS (the benchmark spec's
bound for it) with the same relative term.
"""
import math

import numpy as np

ATOL = 1e-5
U32 = 2.0 ** -24
C_FFT = 0.25
C_OUT = 2.0
ATOL_TC = 1e-3


def rtol_fp32(nchan: int) -> float:
    """Relative per-channel term r(N) of the FP32 tolerance (module docstring)."""
    return (C_FFT * math.log2(nchan) + C_OUT) * U32


def metrics(gpu: np.ndarray, ref: np.ndarray, atol: float = ATOL, rtol: float | None = None) -> dict:
    """Tolerance use (max over channels of error / allowed) and the pure error
    normalised to the RMS. ``ref`` is [nchan, 4] (dual-pol) or [nchan]; rtol
    defaults to r(nchan)."""
    g = np.asarray(gpu, np.float64)
    o = np.asarray(ref, np.float64)
    if rtol is None:
        rtol = rtol_fp32(o.shape[0])
    if o.ndim == 1:
        g, o = g[:, None], o[:, None]
    out = {"ratio": 0.0, "pure": 0.0, "rtol": rtol}
    rms = np.sqrt(np.mean(o ** 2, axis=0))
    for c in range(o.shape[1]):
        err = np.abs(g[:, c] - o[:, c])
        if c < 2:
            scale = rms[c]
            own = np.abs(o[:, c])
        else:
            scale = np.sqrt(rms[0] * rms[1])
            own = np.sqrt(np.abs(o[:, 0] * o[:, 1]))
        allowed = atol * scale + rtol * own
        out["ratio"] = max(out["ratio"], float(np.max(err / allowed)))
        out["pure"] = max(out["pure"], float(np.max(err) / scale))
    return out


def assert_close(gpu, ref, atol: float = ATOL, rtol: float | None = None, what: str = "") -> dict:
    m = metrics(gpu, ref, atol, rtol)
    assert m["ratio"] <= 1.0, f"{what}: error {m['ratio']:.3g}x the tolerance (normalised max {m['pure']:.3g})"
    return m
