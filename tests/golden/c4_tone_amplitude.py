"""Writes the tone amplitude of the precision-stress workload (131072 channels).

The workload asks for a tone 40 dB above the noise floor. Read per channel of
one spectrum: a bin-centred tone of amplitude A gives power A^2 (sum h)^2 and
complex Gaussian noise of per-component sigma gives 2 sigma^2 sum h^2, so
A = 100 * sigma * sqrt(2 sum h^2) / |sum h|. The coefficients come from the
oracle only. Run: python tests/golden/c4_tone_amplitude.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", ".."))
import oracle  # noqa: E402

NCHAN, NTAPS, SIGMA, SNR = 131072, 8, 4.0, 1.0e4


def amplitude() -> float:
    h = oracle.coeffs(NCHAN, NTAPS, oracle.PFB, oracle.WIN_HANN)
    return float(np.sqrt(SNR) * SIGMA * np.sqrt(2.0 * np.sum(h * h)) / abs(np.sum(h)))


if __name__ == "__main__":
    a = amplitude()
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_tone_amplitude.txt"), "w") as f:
        f.write(f"{a!r}\n")
    print(repr(a))
