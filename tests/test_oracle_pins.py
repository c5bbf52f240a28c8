"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's own formulas: each compares the oracle with
an independent algorithm (brute-force DFT), a library routine (numpy FFT,
scipy's window-method FIR design, numpy windows), a closed form (Parseval, the
Dirichlet kernel, the response to impulses and to tones) or a statistical
expectation (noise power), so that a dropped term, a wrong sign, a wrong tap
order or a transposed layout in the oracle fails at least one test.
"""
import numpy as np
import pytest

from paper_1411_0436_gb300 import workloads

PFB, DIRECT = 0, 1
RECT, HANN, HAMMING = 0, 1, 2


def _rand_complex(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def _f64_input(x_pol):
    """Stack per-pol complex series [npol][time] into float64 [time][pol][re, im]."""
    x_pol = np.atleast_2d(x_pol)
    a = np.empty((x_pol.shape[1], x_pol.shape[0], 2), np.float64)
    a[:, :, 0] = x_pol.T.real
    a[:, :, 1] = x_pol.T.imag
    return a


# ---------------------------------------------------------------- FFT (§4) ---

@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256])
def test_fft_matches_bruteforce_dft(oracle_mod, n):
    rng = np.random.default_rng(n)
    x = _rand_complex(rng, n)
    k = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(k, k) / n)  # O(n^2) definition of the DFT
    ref = F @ x
    got = oracle_mod.fft(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [512, 4096, 65536])
def test_fft_matches_numpy(oracle_mod, n):
    rng = np.random.default_rng(7 + n)
    x = _rand_complex(rng, n)
    ref = np.fft.fft(x)
    got = oracle_mod.fft(x)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-12


def test_fft_parseval(oracle_mod):
    rng = np.random.default_rng(3)
    n = 8192
    x = _rand_complex(rng, n)
    X = oracle_mod.fft(x)
    assert abs(np.sum(np.abs(X) ** 2) - n * np.sum(np.abs(x) ** 2)) <= 1e-12 * n * np.sum(np.abs(x) ** 2)


def test_fft_rejects_non_power_of_two(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.fft(np.zeros(12, np.complex128))


# ------------------------------------------------------- coefficients (§4) ---

@pytest.mark.parametrize("nchan,ntaps", [(64, 8), (1024, 8), (256, 4), (128, 16)])
@pytest.mark.parametrize("window,name", [(HANN, "hann"), (HAMMING, "hamming"), (RECT, "boxcar")])
def test_pfb_coeffs_match_scipy_firwin(oracle_mod, nchan, ntaps, window, name):
    """Window-method low-pass of cutoff half a channel: scipy.signal.firwin."""
    signal = pytest.importorskip("scipy.signal")
    L = nchan * ntaps
    ref = nchan * signal.firwin(L, 1.0 / nchan, window=name, scale=False)
    got = oracle_mod.coeffs(nchan, ntaps, PFB, window)
    assert got.shape == (L,)
    assert np.max(np.abs(got - ref)) <= 1e-12


@pytest.mark.parametrize("window,fn", [(HANN, np.hanning), (HAMMING, np.hamming),
                                       (RECT, np.ones)])
def test_direct_coeffs_are_the_window(oracle_mod, window, fn):
    n = 512
    got = oracle_mod.coeffs(n, 1, DIRECT, window)
    assert np.max(np.abs(got - fn(n))) <= 1e-14


def test_pfb_coeffs_symmetric_and_half_power_at_channel_edge(oracle_mod):
    """A linear-phase low-pass whose amplitude falls to 1/2 half a channel out."""
    n, P = 256, 8
    h = oracle_mod.coeffs(n, P, PFB, HANN)
    assert np.max(np.abs(h - h[::-1])) <= 1e-15
    i = np.arange(h.size)

    def resp(delta):  # DTFT at delta channels from DC
        return abs(np.sum(h * np.exp(-2j * np.pi * delta * i / n)))

    H0 = resp(0.0)
    assert abs(resp(0.5) / H0 - 0.5) < 0.01
    assert resp(0.25) / H0 > 0.9
    assert resp(1.5) / H0 < 1e-2


# --------------------------------------------------- pre-filter (§4, PFB) ---

@pytest.mark.parametrize("mode,P", [(PFB, 8), (PFB, 3), (DIRECT, 1)])
def test_fir_impulse_reproduces_coefficients(oracle_mod, mode, P):
    """Tap order: h[t*N + n] multiplies frame s + t (the oldest frame is t = 0)."""
    n, npol, pol = 32, 2, 1
    t0, n0 = P + 1, 5
    S = t0 + 2
    x = np.zeros(((S + P - 1) * n, npol), np.complex128)
    v = 3.0 - 2.0j
    x[t0 * n + n0, pol] = v
    h = oracle_mod.coeffs(n, P, mode, HANN)
    xin = _f64_input(x.T)
    for s in range(S):
        y = oracle_mod.fir(xin, n, P, npol, s, pol, mode, HANN)
        expect = np.zeros(n, np.complex128)
        t = t0 - s
        if 0 <= t < (P if mode == PFB else 1):
            expect[n0] = v * h[t * n + n0]
        assert np.array_equal(y, expect), (s, y[n0], expect[n0])
        assert np.all(oracle_mod.fir(xin, n, P, npol, s, 0, mode, HANN) == 0)


# ---------------------------------------- whole path: detect + accumulate ---

@pytest.mark.parametrize("v", [(1, 0), (-128, 0), (127, -128), (-7, 3), (0, 1)])
def test_impulse_gives_flat_exact_power(oracle_mod, v):
    """Direct mode, impulse at the first sample: |X[k]|^2 = |v|^2 for every k."""
    n = 64
    x = np.zeros((n, 2, 2), np.int8)
    x[0, 0] = v
    x[0, 1] = (v[1], v[0])
    out = oracle_mod.channelize(x, n, 1, 2, 1, DIRECT, RECT)
    p = float(v[0]) ** 2 + float(v[1]) ** 2
    assert np.all(out[:, 0] == p) and np.all(out[:, 1] == p)


def test_impulse_offset_gives_flat_power(oracle_mod):
    n = 128
    x = np.zeros((n, 1, 2), np.int8)
    x[37, 0] = (5, -9)
    out = oracle_mod.channelize(x, n, 1, 1, 1, DIRECT, RECT)
    assert np.max(np.abs(out - 106.0)) <= 1e-12


def test_pfb_impulse_gives_flat_sum_of_squared_taps(oracle_mod):
    n, P = 64, 8
    t0, n0 = 9, 21
    S = 20
    x = np.zeros(((S + P - 1) * n, 1, 2), np.int8)
    x[t0 * n + n0, 0] = (4, 3)
    h = oracle_mod.coeffs(n, P, PFB, HANN)
    expect = 25.0 * np.sum(h[n0::n] ** 2)  # all P spectra that see the impulse
    out = oracle_mod.channelize(x, n, P, 1, S, PFB, HANN)
    assert np.max(np.abs(out - expect)) <= 1e-12 * expect


def _tone(n, S, P, k, amp, npol=1):
    m = np.arange((S + P - 1) * n)
    t = amp * np.exp(2j * np.pi * k * m / n)
    return _f64_input(np.vstack([t] * npol))


@pytest.mark.parametrize("k0", [0, 1, 17, 100, 255])
def test_direct_tone_lands_in_its_bin(oracle_mod, k0):
    n, S, A = 256, 3, 2.5
    out = oracle_mod.channelize_f64(_tone(n, S, 1, k0, A), n, 1, 1, S, DIRECT, RECT)
    peak = S * (n * A) ** 2
    assert abs(out[k0] - peak) <= 1e-12 * peak
    assert int(np.argmax(out)) == k0
    others = np.delete(out, k0)
    assert np.max(others) <= 1e-20 * peak


@pytest.mark.parametrize("k0", [3, 64])
def test_pfb_tone_matches_polyphase_gain(oracle_mod, k0):
    """PFB tone at an integer bin: X[k] = A * G[k - k0], G the DFT of the
    polyphase sum g[n] = sum_t h[t*N + n]; in particular X[k0] = A sum h."""
    n, P, S, A = 128, 8, 4, 1.5
    h = oracle_mod.coeffs(n, P, PFB, HANN)
    g = h.reshape(P, n).sum(0)
    G = np.fft.fft(g)
    expect = S * A * A * np.abs(np.roll(G, k0)) ** 2
    out = oracle_mod.channelize_f64(_tone(n, S, P, k0, A), n, P, 1, S, PFB, HANN)
    assert abs(out[k0] - S * (A * h.sum()) ** 2) <= 1e-12 * out[k0]
    assert np.max(np.abs(out - expect)) <= 1e-11 * np.max(expect)


@pytest.mark.parametrize("delta", [0.4, -0.6, 0.25])
def test_direct_scalloping_is_dirichlet(oracle_mod, delta):
    n, S, A, k0 = 256, 2, 1.0, 40
    out = oracle_mod.channelize_f64(_tone(n, S, 1, k0 + delta, A), n, 1, 1, S, DIRECT, RECT)
    expect = S * A * A * np.sin(np.pi * delta) ** 2 / np.sin(np.pi * delta / n) ** 2
    assert abs(out[k0] - expect) <= 1e-10 * expect


@pytest.mark.parametrize("delta", [0.4, -0.6])
def test_pfb_scalloping_is_coefficient_dtft(oracle_mod, delta):
    n, P, S, A, k0 = 128, 8, 3, 1.0, 23
    h = oracle_mod.coeffs(n, P, PFB, HANN)
    i = np.arange(h.size)
    expect = S * A * A * abs(np.sum(h * np.exp(2j * np.pi * delta * i / n))) ** 2
    out = oracle_mod.channelize_f64(_tone(n, S, P, k0 + delta, A), n, P, 1, S, PFB, HANN)
    assert abs(out[k0] - expect) <= 1e-10 * expect


def test_cross_products_follow_x_times_conj_y(oracle_mod):
    """Y = i X gives X conj(Y) = -i |X|^2: Re = 0, Im = -XX, YY = XX."""
    n, S = 64, 5
    rng = np.random.default_rng(11)
    a = rng.integers(-100, 100, size=(S * n, 2)).astype(np.int8)
    x = np.empty((S * n, 2, 2), np.int8)
    x[:, 0] = a
    x[:, 1, 0] = -a[:, 1]
    x[:, 1, 1] = a[:, 0]
    out = oracle_mod.channelize(x, n, 1, 2, S, DIRECT, RECT)
    XX, YY, XYr, XYi = out.T
    assert np.max(np.abs(YY - XX)) <= 1e-12 * XX.max()
    assert np.max(np.abs(XYr)) <= 1e-12 * XX.max()
    assert np.max(np.abs(XYi + XX)) <= 1e-12 * XX.max()


def test_polarisation_layout_is_interleaved(oracle_mod):
    """Samples are [time][pol][re, im]: energy in pol 1 only shows in YY only."""
    n, S = 32, 2
    rng = np.random.default_rng(5)
    x = np.zeros((S * n, 2, 2), np.int8)
    x[:, 1] = rng.integers(-50, 50, size=(S * n, 2))
    out = oracle_mod.channelize(x, n, 1, 2, S, DIRECT, RECT)
    assert np.all(out[:, 0] == 0) and np.all(out[:, 2] == 0) and np.all(out[:, 3] == 0)
    assert np.all(out[:, 1] > 0)


def test_accumulation_is_a_plain_sum_over_spectra(oracle_mod):
    n, P, S = 64, 8, 9
    rng = np.random.default_rng(21)
    x = rng.integers(-127, 128, size=((S + P - 1) * n, 2, 2)).astype(np.int8)
    total = oracle_mod.channelize(x, n, P, 2, S, PFB, HANN)
    parts = sum(oracle_mod.channelize(x[s * n:], n, P, 2, 1, PFB, HANN) for s in range(S))
    assert np.max(np.abs(total - parts)) <= 1e-12 * np.max(np.abs(total))


def test_dual_pol_xx_matches_single_pol(oracle_mod):
    n, P, S = 128, 8, 6
    rng = np.random.default_rng(8)
    x = rng.integers(-127, 128, size=((S + P - 1) * n, 2, 2)).astype(np.int8)
    dual = oracle_mod.channelize(x, n, P, 2, S, PFB, HANN)
    single = oracle_mod.channelize(np.ascontiguousarray(x[:, :1]), n, P, 1, S, PFB, HANN)
    single_y = oracle_mod.channelize(np.ascontiguousarray(x[:, 1:]), n, P, 1, S, PFB, HANN)
    assert np.max(np.abs(dual[:, 0] - single)) <= 1e-13 * single.max()
    assert np.max(np.abs(dual[:, 1] - single_y)) <= 1e-13 * single_y.max()


def test_thread_count_does_not_change_result(oracle_mod):
    n, P, S = 256, 8, 13
    rng = np.random.default_rng(4)
    x = rng.integers(-127, 128, size=((S + P - 1) * n, 2, 2)).astype(np.int8)
    a = oracle_mod.channelize(x, n, P, 2, S, PFB, HANN, nthreads=1)
    b = oracle_mod.channelize(x, n, P, 2, S, PFB, HANN, nthreads=4)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


# ------------------------------------------------------------- statistics ---

@pytest.mark.parametrize("mode,P,window", [(DIRECT, 1, RECT), (PFB, 8, HANN)])
def test_gaussian_noise_power_and_correlation(oracle_mod, mode, P, window):
    """E[XX] = E[YY] = 2 sigma^2 sum h^2, E[Re XY*] = rho * that, E[Im XY*] = 0;
    the spectrum is flat within the chi-square scatter of the average."""
    n, S, sigma, rho = 256, 400, 3.0, 0.3
    rng = np.random.default_rng(99)
    T = (S + P - 1) * n
    g0 = sigma * _rand_complex(rng, T)
    g1 = sigma * _rand_complex(rng, T)
    y = rho * g0 + np.sqrt(1 - rho * rho) * g1
    out = oracle_mod.channelize_f64(_f64_input(np.vstack([g0, y])), n, P, 2, S, mode, window) / S
    h = oracle_mod.coeffs(n, P, mode, window)
    mu = 2 * sigma ** 2 * np.sum(h * h)
    s_eff = S / (2.0 if mode == PFB else 1.0)  # overlapping PFB frames correlate spectra
    tol_mean = 6.0 / np.sqrt(n * s_eff)
    for c in (0, 1):
        assert abs(out[:, c].mean() / mu - 1.0) < tol_mean
        assert np.max(np.abs(out[:, c] / mu - 1.0)) < 6.0 / np.sqrt(s_eff)
    assert abs(out[:, 2].mean() / (rho * mu) - 1.0) < 8.0 / (rho * np.sqrt(n * s_eff))
    assert abs(out[:, 3].mean() / mu) < 6.0 / np.sqrt(n * s_eff)


def test_int8_noise_power_includes_rounding(oracle_mod):
    """Rounding to integers adds 1/12 to each component's variance."""
    bank = workloads.Bank(512, 1, 2, DIRECT, RECT, 200, sigma=6.0)
    x = workloads.generate(bank, 1234)
    out = oracle_mod.channelize(x, bank.nchan, 1, 2, bank.nspectra, DIRECT, RECT) / bank.nspectra
    mu = 2 * (6.0 ** 2 + 1.0 / 12.0) * bank.nchan
    tol = 6.0 / np.sqrt(bank.nchan * bank.nspectra)
    assert abs(out[:, 0].mean() / mu - 1.0) < tol
    assert abs(out[:, 1].mean() / mu - 1.0) < tol


def test_c4_tone_amplitude_fixture(oracle_mod):
    """The stored precision-stress amplitude gives 40 dB per-channel SNR."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "c4_tone_amplitude.txt")
    stored = float(open(path).read())
    assert stored == workloads.C4_TONE_AMP
    h = oracle_mod.coeffs(131072, 8, PFB, HANN)
    snr = stored ** 2 * h.sum() ** 2 / (2 * 4.0 ** 2 * np.sum(h * h))
    assert abs(snr / 1e4 - 1) < 1e-12
