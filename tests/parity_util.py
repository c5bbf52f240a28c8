"""Comparison of the CUDA path's accumulated spectra with the FP64 oracle.

Tolerance (per channel k, after S spectra):
  auto terms XX, YY:   |G_k - O_k| <= ATOL * RMS(O) + rtol * |O_k|
  cross terms Re, Im:  |G_k - O_k| <= ATOL * sqrt(RMS(XX) RMS(YY))
                                      + rtol * sqrt(XX_k YY_k)
ATOL = 1e-5 is the error normalised to the spectrum RMS that the FP32 path
must meet. The rtol term is the FP32 rounding of the channel's own value:
a channel whose power T is far above the RMS (a tone) carries a rounding
error of order u * T with u = 2^-24 however the arithmetic is ordered, and
this can exceed 1e-5 * RMS when T / RMS reaches ~100. rtol is 64 u (about
3.8e-6) for the FP32 path. The pure normalised error max_k |G - O| / RMS is
reported alongside.
"""
import numpy as np

ATOL = 1e-5
U32 = 2.0 ** -24
RTOL_FP32 = 64 * U32
# Tensor-core path (first DFT pass with bf16 hi/lo operands, about 16
# significant bits): 1e-3 of the spectrum RMS, plus 64 units of 2^-17 of the
# channel's own value.
ATOL_TC = 1e-3
RTOL_TC = 64 * 2.0 ** -17


def metrics(gpu: np.ndarray, ref: np.ndarray, atol: float = ATOL, rtol: float = RTOL_FP32) -> dict:
    g = np.asarray(gpu, np.float64)
    o = np.asarray(ref, np.float64)
    if o.ndim == 1:
        g, o = g[:, None], o[:, None]
    out = {"ratio": 0.0, "pure": 0.0}
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


def assert_close(gpu, ref, atol: float = ATOL, rtol: float = RTOL_FP32, what: str = "") -> dict:
    m = metrics(gpu, ref, atol, rtol)
    assert m["ratio"] <= 1.0, f"{what}: error {m['ratio']:.3g}x the tolerance (normalised max {m['pure']:.3g})"
    return m
