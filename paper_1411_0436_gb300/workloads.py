"""Seeded synthetic inputs shaped like the spectrometer workloads of arXiv 1411.0436.

This module only draws input samples: Gaussian voltages, optional
polarisation correlation and injected tones, rounded and clipped to int8 in
the [time][pol][re, im] layout. It holds none of the channelizer's arithmetic
and is shared by the tests, the benchmark and the CPU oracle's callers.

The paper's own inputs (GBT observations, §4.1; disk files, §5) are not
available; the recipes below stand in for them with the same sample format
(8-bit complex, dual polarisation, §4) and the channel counts of the VEGAS
heterogeneous modes (Table 1) and of the benchmark (2^16 and 2^20 points, §5).
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import os
from typing import Sequence, Tuple

import numpy as np

PFB, DIRECT = 0, 1
WIN_RECT, WIN_HANN, WIN_HAMMING = 0, 1, 2

SEED_BASE = 14110436
BLOCK = 1 << 20  # time samples drawn per generator call; part of the recipe


@dataclasses.dataclass(frozen=True)
class Tone:
    """Complex tone amp * exp(2 pi i * bin * m / nchan) added to the listed pols."""
    amp: float
    bin: float
    pols: Tuple[int, ...] = (0, 1)


@dataclasses.dataclass(frozen=True)
class Bank:
    """One channelizer problem: plan parameters plus the input recipe."""
    nchan: int
    ntaps: int
    npol: int
    mode: int
    window: int
    nspectra: int
    sigma: float = 20.0
    rho: float = 0.0
    tones: Tuple[Tone, ...] = ()

    @property
    def taps_used(self) -> int:
        return 1 if self.mode == DIRECT else self.ntaps

    @property
    def nsamples(self) -> int:
        """Time samples per polarisation the input must hold."""
        return (self.nspectra + self.taps_used - 1) * self.nchan

    @property
    def nbytes(self) -> int:
        return self.nsamples * self.npol * 2

    def with_spectra(self, nspectra: int) -> "Bank":
        return dataclasses.replace(self, nspectra=nspectra)


# Tone amplitude of the precision-stress workload: the per-channel SNR of one
# spectrum, A^2 (sum h)^2 / (2 sigma^2 sum h^2), equals 1e4 (40 dB) for a
# bin-centred tone with sigma = 4 and the 8-tap Hann-windowed sinc at 131072
# channels. Written by tests/golden/c4_tone_amplitude.py from the oracle's
# coefficients.
C4_TONE_AMP = 1.4784316925310972

CONFIGS = {
    # Single-pol PFB, 1024 channels, 8 taps, 64 spectra, tone at bin 123.4.
    "c1": (Bank(1024, 8, 1, PFB, WIN_HANN, 64, 20.0, 0.0, (Tone(30.0, 123.4, (0,)),)),),
    # Dual-pol PFB, 32768 channels, 8 taps, 1000 spectra, X/Y correlation 0.3,
    # one tone in both pols and one in X only.
    "c2": (Bank(32768, 8, 2, PFB, WIN_HANN, 1000, 20.0, 0.3,
                (Tone(30.0, 0.1 * 32768 + 0.25, (0, 1)), Tone(20.0, 0.37 * 32768 + 0.5, (0,)))),),
    # Dual-pol direct FFT, 524288 channels, 256 spectra.
    "c3": (Bank(524288, 1, 2, DIRECT, WIN_RECT, 256, 20.0),),
    # Precision stress: dual-pol PFB, 131072 channels, 4096 spectra, sigma 4,
    # a bin-centred tone 40 dB above the per-channel noise floor.
    "c4": (Bank(131072, 8, 2, PFB, WIN_HANN, 4096, 4.0, 0.0,
                (Tone(C4_TONE_AMP, 0.2 * 131072, (0, 1)),)),),
    # Batched multi-beam: 8 banks, PFB and direct alternating, uneven integrations.
    "c5": tuple(
        Bank(n, 8 if i % 2 == 0 else 1, 2, PFB if i % 2 == 0 else DIRECT,
             WIN_HANN if i % 2 == 0 else WIN_RECT, s, 20.0)
        for i, (n, s) in enumerate(zip(
            (1024, 4096, 16384, 32768, 65536, 131072, 262144, 524288),
            (2048, 1024, 1024, 512, 256, 128, 64, 64)))
    ),
}

CONFIG_INDEX = {"c1": 0, "c2": 1, "c3": 2, "c4": 3, "c5": 4}


def _fill_block(bank: Bank, seed: int, i: int, m0: int, b: int, tables, out) -> None:
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, i])))
    g = rng.standard_normal((b, bank.npol, 2), dtype=np.float32)
    g *= np.float32(bank.sigma)
    if bank.npol == 2 and bank.rho != 0.0:
        c = np.float32(np.sqrt(max(0.0, 1.0 - bank.rho * bank.rho)))
        g[:, 1, :] = np.float32(bank.rho) * g[:, 0, :] + c * g[:, 1, :]
    for t, tab in zip(bank.tones, tables):
        start = np.exp(2j * np.pi * np.mod(t.bin * m0, bank.nchan) / bank.nchan)
        ph = (t.amp * start) * tab[:b]
        re, im = ph.real.astype(np.float32), ph.imag.astype(np.float32)
        for p in t.pols:
            if p < bank.npol:
                g[:, p, 0] += re
                g[:, p, 1] += im
    np.rint(g, out=g)
    np.clip(g, -127, 127, out=g)
    out[m0:m0 + b] = g.astype(np.int8)


def generate(bank: Bank, seed: int, nsamples: int | None = None,
             threads: int | None = None) -> np.ndarray:
    """Draw int8 samples of shape [time, npol, 2] for ``bank``.

    Recipe: the time axis is cut into blocks of BLOCK samples; block i draws
    float32 standard normals of shape [block, npol, 2] from its own PCG64
    stream, seeded by SeedSequence([seed, i]), scaled by sigma; pol 1 is
    rho * g0 + sqrt(1 - rho^2) * g1; each tone is the float64 phasor
    amp * exp(2 pi i bin m / nchan), formed as the block's start phasor times a
    per-offset table, and added in float32; the sum is rounded half-to-even and
    clipped to [-127, 127]. The result does not depend on ``threads``.
    """
    n = bank.nsamples if nsamples is None else nsamples
    out = np.empty((n, bank.npol, 2), np.int8)
    offs = np.arange(min(BLOCK, n), dtype=np.float64)
    tables = [np.exp(2j * np.pi * np.mod((t.bin / bank.nchan) * offs, 1.0)) for t in bank.tones]
    starts = list(range(0, n, BLOCK))
    work = [(i, m0, min(BLOCK, n - m0)) for i, m0 in enumerate(starts)]
    nthr = threads if threads is not None else min(16, os.cpu_count() or 1)
    if nthr <= 1 or len(work) <= 1:
        for i, m0, b in work:
            _fill_block(bank, seed, i, m0, b, tables, out)
    else:
        with concurrent.futures.ThreadPoolExecutor(nthr) as ex:
            list(ex.map(lambda w: _fill_block(bank, seed, w[0], w[1], w[2], tables, out), work))
    return out


def config_banks(name: str) -> Sequence[Bank]:
    return CONFIGS[name]


def config_seed(name: str, bank_index: int = 0) -> int:
    return SEED_BASE + CONFIG_INDEX[name] + 100 * bank_index
