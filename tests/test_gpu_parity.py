"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Inputs come from the shared seeded generators; the oracle never sees anything
the CUDA path produced. Sizes are chosen so the oracle finishes in seconds
while the GPU runs span several tiles, several scratch chunks and ragged
tails; the full workload sizes are in test_gpu_workloads.py.
"""
import numpy as np
import pytest

from parity_util import U32, assert_close
from paper_1411_0436_gb300 import workloads
from paper_1411_0436_gb300.workloads import DIRECT, PFB, WIN_HAMMING, WIN_HANN, WIN_RECT, Bank, Tone

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run_gpu(bank: Bank, x: np.ndarray, repeat: int = 1, flags: int = 0, tuning=None) -> np.ndarray:
    from paper_1411_0436_gb300.vspec import Plan
    with Plan(bank.nchan, bank.ntaps, bank.npol, bank.mode, bank.window, flags) as plan:
        if tuning:
            plan.tune(**tuning)
        d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8).reshape(-1)).cuda()
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        for _ in range(repeat):
            plan.execute(d_in, bank.nspectra, acc)
        torch.cuda.synchronize()
        out = acc.cpu().numpy().astype(np.float64)
    return out.reshape(bank.nchan, 4) if bank.npol == 2 else out


def run_oracle(oracle_mod, bank: Bank, x: np.ndarray) -> np.ndarray:
    return oracle_mod.channelize(x, bank.nchan, bank.ntaps, bank.npol, bank.nspectra,
                                 bank.mode, bank.window)


SMALL = [
    # nchan, ntaps, npol, mode, window, nspectra
    (16, 8, 2, PFB, WIN_HANN, 5),
    (16, 1, 1, DIRECT, WIN_RECT, 3),
    (64, 8, 1, PFB, WIN_HANN, 9),
    (256, 8, 2, PFB, WIN_HANN, 17),
    (256, 3, 2, PFB, WIN_HAMMING, 11),
    (512, 16, 2, PFB, WIN_HANN, 20),
    (1024, 8, 1, PFB, WIN_HANN, 64),
    (1024, 5, 2, PFB, WIN_RECT, 13),
    (2048, 8, 2, PFB, WIN_HANN, 33),
    (4096, 1, 2, DIRECT, WIN_RECT, 9),
    (4096, 8, 2, PFB, WIN_HANN, 19),
    (8192, 2, 1, PFB, WIN_HANN, 7),
    (8192, 1, 2, DIRECT, WIN_HANN, 6),
    (16384, 8, 2, PFB, WIN_HANN, 10),
    (32768, 8, 2, PFB, WIN_HANN, 67),   # ragged: not a multiple of the clusters or tiles
    (32768, 8, 2, PFB, WIN_HANN, 1),    # fewer spectra than clusters
    (32768, 1, 2, DIRECT, WIN_HANN, 23),
    (2048, 1, 2, DIRECT, WIN_RECT, 40),
    (16384, 8, 2, PFB, WIN_HAMMING, 300),
    (32768, 12, 2, PFB, WIN_HAMMING, 5),
    (65536, 8, 2, PFB, WIN_HANN, 4),
    (65536, 4, 1, PFB, WIN_HANN, 6),
    (131072, 1, 2, DIRECT, WIN_RECT, 3),
    (262144, 8, 2, PFB, WIN_HANN, 2),
    (524288, 1, 2, DIRECT, WIN_RECT, 2),
    (1 << 20, 1, 2, DIRECT, WIN_RECT, 1),
    (1 << 19, 8, 2, PFB, WIN_HANN, 3),     # taps read from the input (no register window)
    (1 << 20, 8, 2, PFB, WIN_HAMMING, 2),
    (1 << 20, 16, 1, PFB, WIN_HANN, 2),
    (1 << 20, 1, 1, DIRECT, WIN_RECT, 2),  # single-pol, 32-byte column segments
    (1 << 18, 16, 2, PFB, WIN_HANN, 3),
    # register-column kernel A: every column shape, windows, fewer taps than
    # the register window (leading zero taps)
    (8192, 8, 2, PFB, WIN_HANN, 9),        # 4-point columns, two per thread
    (32768, 5, 2, PFB, WIN_RECT, 9),       # 16-point columns, 3 zero taps
    (131072, 8, 2, PFB, WIN_HANN, 5),      # 64-point columns, passes 8 x 8
    (262144, 6, 2, PFB, WIN_HAMMING, 3),   # 128-point columns, 4-sample tile rows
    (16384, 1, 2, DIRECT, WIN_HANN, 17),   # direct, 8-point columns, window
    (65536, 1, 2, DIRECT, WIN_HAMMING, 5), # direct, passes 16 x 2, window
    (262144, 1, 2, DIRECT, WIN_HANN, 3),   # direct, passes 16 x 8, window
    # one-row transforms: frame ring with the most taps, and with one
    (1024, 16, 2, PFB, WIN_HANN, 21),
    (512, 1, 1, DIRECT, WIN_HAMMING, 7),
]


def fused_applies(n, p, npol, mode):
    """Sizes where a default plan takes the one-pass fused cluster path."""
    return npol == 2 and 2048 <= n <= 32768 and (mode == DIRECT or p == 8)


@pytest.mark.parametrize("cfg", SMALL, ids=lambda c: f"N{c[0]}_P{c[1]}_pol{c[2]}_m{c[3]}_w{c[4]}_S{c[5]}")
def test_matches_oracle(oracle_mod, cfg):
    from paper_1411_0436_gb300.vspec import PLAN_TWO_KERNEL
    n, p, npol, mode, win, s = cfg
    tones = (Tone(25.0, n * 0.3 + 0.4, (0, 1)),) if n >= 64 else ()
    bank = Bank(n, p, npol, mode, win, s, sigma=20.0, rho=0.3 if npol == 2 else 0.0, tones=tones)
    x = workloads.generate(bank, 1000 + n + p)
    o = run_oracle(oracle_mod, bank, x)
    assert_close(run_gpu(bank, x), o, what=str(cfg))
    if fused_applies(n, p, npol, mode):  # the one-pass fused path alone, and the general path
        from paper_1411_0436_gb300.vspec import NEVER
        assert_close(run_gpu(bank, x, tuning={"two_kernel_from": NEVER, "assist_permille": 0}), o,
                     what=f"{cfg} fused")
        assert_close(run_gpu(bank, x, flags=PLAN_TWO_KERNEL), o, what=f"{cfg} two-kernel")


def test_impulse_is_bit_exact_for_every_int8_value():
    """Direct mode, impulse at the first sample: every channel is exactly
    |v|^2 (and the cross terms are exact integers), which pins the int8 unpack."""
    n = 64
    bank = Bank(n, 1, 2, DIRECT, WIN_RECT, 1)
    for v in range(-128, 128):
        x = np.zeros((n, 2, 2), np.int8)
        x[0, 0] = (v, 127)    # X[k] = v + 127 i
        x[0, 1] = (-128, v)   # Y[k] = -128 + v i
        g = run_gpu(bank, x)
        expect = np.array([v * v + 127 * 127, 128 * 128 + v * v,
                           -128 * v + 127 * v, 127 * -128 - v * v], np.float64)
        assert np.array_equal(g, np.broadcast_to(expect, g.shape)), v


@pytest.mark.parametrize("n,k0", [(1024, 123), (32768, 3277), (32768, 0), (131072, 26214)])
def test_tone_lands_in_its_channel(oracle_mod, n, k0):
    """Channel indexing: a strong tone at an integer bin is the argmax (same bin
    as the oracle), bit-exact as an index."""
    bank = Bank(n, 8, 2, PFB, WIN_HANN, 3, sigma=5.0, tones=(Tone(60.0, float(k0), (0, 1)),))
    x = workloads.generate(bank, 7 + k0)
    g = run_gpu(bank, x)
    o = run_oracle(oracle_mod, bank, x)
    assert int(np.argmax(g[:, 0])) == k0 == int(np.argmax(o[:, 0]))
    assert int(np.argmax(g[:, 1])) == k0


def test_accumulates_and_dump_clears():
    from paper_1411_0436_gb300.vspec import Plan
    bank = Bank(4096, 8, 2, PFB, WIN_HANN, 5)
    x = workloads.generate(bank, 3)
    once = run_gpu(bank, x)
    with Plan(bank.nchan, bank.ntaps, bank.npol, bank.mode, bank.window) as plan:
        d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        plan.execute(d_in, bank.nspectra, acc)
        plan.execute(d_in, bank.nspectra, acc)
        h = torch.empty(plan.out_floats, dtype=torch.float32).pin_memory()
        plan.dump(acc, h)
        torch.cuda.synchronize()
        twice = h.numpy().astype(np.float64).reshape(-1, 4)
        assert torch.count_nonzero(acc).item() == 0
        plan.execute(d_in, 0, acc)  # no-op
        torch.cuda.synchronize()
        assert torch.count_nonzero(acc).item() == 0
    # the second call adds the same partials again: doubling is exact in FP32
    assert np.max(np.abs(twice - 2 * once)) <= 2 * U32 * np.max(np.abs(twice))


def test_repeat_runs_are_bitwise_identical():
    bank = Bank(32768, 8, 2, PFB, WIN_HANN, 70, rho=0.3)
    x = workloads.generate(bank, 11)
    a = run_gpu(bank, x)
    b = run_gpu(bank, x)
    assert np.array_equal(a, b)


def test_streaming_calls_equal_one_call(oracle_mod):
    """Consecutive calls over inputs overlapped by (P-1)*N samples add up to
    one call over the whole run (the paper's per-iteration loop)."""
    from paper_1411_0436_gb300.vspec import Plan
    bank = Bank(8192, 8, 2, PFB, WIN_HANN, 24, rho=0.3)
    x = workloads.generate(bank, 21)
    whole = run_gpu(bank, x)
    n, P = bank.nchan, bank.ntaps
    with Plan(n, P, 2, PFB, WIN_HANN) as plan:
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        for s0, cnt in [(0, 10), (10, 9), (19, 5)]:
            part = np.ascontiguousarray(x[s0 * n:(s0 + cnt + P - 1) * n])
            plan.execute(torch.from_numpy(part.view(np.uint8).reshape(-1)).cuda(), cnt, acc)
        torch.cuda.synchronize()
        got = acc.cpu().numpy().astype(np.float64).reshape(-1, 4)
    assert_close(got, run_oracle(oracle_mod, bank, x))
    assert_close(got, whole)


def test_error_paths_on_device():
    from paper_1411_0436_gb300 import vspec
    with vspec.Plan(1024, 8, 2, PFB, WIN_HANN) as plan:
        buf = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
        acc = torch.zeros(4096, dtype=torch.float32, device="cuda")
        lib = vspec.load()
        s = torch.cuda.current_stream().cuda_stream
        assert lib.vspec_execute(plan.handle, buf.data_ptr() + 4, 1, acc.data_ptr(), s) == vspec.ERR_ALIGNMENT
        assert lib.vspec_execute(plan.handle, buf.data_ptr(), 1, acc.data_ptr() + 4, s) == vspec.ERR_ALIGNMENT
        assert lib.vspec_execute(plan.handle, buf.data_ptr(), -1, acc.data_ptr(), s) == vspec.ERR_INVALID_ARG
        assert lib.vspec_dump(plan.handle, acc.data_ptr() + 8, None, s) == vspec.ERR_ALIGNMENT
        sb, hp = plan.info()
        assert sb > 0 and hp == 1  # one-row transform: FIR, FFT and detection in one kernel
    with vspec.Plan(131072, 8, 2, PFB, WIN_HANN) as plan:
        assert plan.info()[1] == 2  # 4 GiB chunk scratch: the intermediate goes through HBM
        plan.tune(chunk_spectra=16)  # 32 MiB chunks stay in L2
        assert plan.info()[1] == 1
    with vspec.Plan(32768, 8, 2, PFB, WIN_HANN) as plan:
        assert plan.info()[1] == 2  # long calls switch to the two-kernel path
        plan.tune(two_kernel_from=vspec.NEVER)
        assert plan.info()[1] == 1  # one-pass fused path only


@pytest.mark.parametrize("cfg", [(32768, 8, 2, PFB, WIN_HANN, 300), (1024, 8, 1, PFB, WIN_HANN, 70),
                                 (131072, 1, 2, DIRECT, WIN_RECT, 40)])
def test_execute_host_pipeline_matches_oracle(oracle_mod, cfg):
    """Host input -> host output (the paper's copy / compute / copy loop), in
    every input mode: staged chunks with overlapped copies, pinned input read
    directly by the kernels (mapped), the automatic choice for pinned and for
    pageable input; a second call must overwrite, not add to, the output."""
    from paper_1411_0436_gb300.vspec import HOST_AUTO, HOST_MAPPED, HOST_STAGED, Plan
    n, p, npol, mode, win, s = cfg
    bank = Bank(n, p, npol, mode, win, s, rho=0.3 if npol == 2 else 0.0,
                tones=(Tone(25.0, n * 0.21 + 0.3, (0,)),))
    x = workloads.generate(bank, 77 + n)
    o = run_oracle(oracle_mod, bank, x)
    pinned = torch.from_numpy(x.view(np.uint8).reshape(-1)).pin_memory()
    pageable = np.ascontiguousarray(x.view(np.uint8).reshape(-1))
    with Plan(n, p, npol, mode, win) as plan:
        h_out = torch.empty(plan.out_floats, dtype=torch.float32).pin_memory()
        for host_mode, h_in, chunk in ((HOST_STAGED, pinned, 0), (HOST_STAGED, pinned, 1 << 20),
                                       (HOST_MAPPED, pinned, 0), (HOST_AUTO, pinned, 0),
                                       (HOST_AUTO, pageable, 0)):
            plan.set_host_mode(host_mode, chunk)
            for _ in range(2):
                h_out.fill_(123.0)
                plan.execute_host(h_in, s, h_out)
                torch.cuda.synchronize()
                got = h_out.numpy().astype(np.float64)
                assert_close(got.reshape(o.shape), o, what=f"{cfg} host mode {host_mode}")


def test_mapped_host_mode_rejects_pageable_input():
    from paper_1411_0436_gb300 import vspec
    with vspec.Plan(4096, 8, 2, PFB, WIN_HANN) as plan:
        plan.set_host_mode(vspec.HOST_MAPPED)
        h_in = np.zeros(4096 * 4 * 9, np.uint8)  # pageable
        h_out = np.zeros(4096 * 4, np.float32)
        with pytest.raises(vspec.VspecError) as e:
            plan.execute_host(h_in, 2, h_out)
        assert e.value.status == vspec.ERR_INVALID_ARG
        with pytest.raises(vspec.VspecError):
            plan.set_host_mode(3)
        with pytest.raises(vspec.VspecError):
            plan.set_host_mode(vspec.HOST_STAGED, 1000)  # below 1 MiB


def test_batch_graph_matches_single_banks(oracle_mod):
    """Banks of different sizes and modes in one CUDA-graph launch give what
    one plan per bank gives; replays and re-captures (new pointers) agree."""
    from paper_1411_0436_gb300.vspec import Batch
    banks = [Bank(1024, 8, 2, PFB, WIN_HANN, 40), Bank(4096, 1, 2, DIRECT, WIN_RECT, 20),
             Bank(16384, 8, 2, PFB, WIN_HANN, 12), Bank(32768, 8, 2, PFB, WIN_HANN, 9),
             Bank(65536, 1, 2, DIRECT, WIN_RECT, 4), Bank(2048, 8, 1, PFB, WIN_HAMMING, 30)]
    xs = [workloads.generate(b, 500 + i) for i, b in enumerate(banks)]
    refs = [run_oracle(oracle_mod, b, x) for b, x in zip(banks, xs)]
    with Batch([(b.nchan, b.ntaps, b.npol, b.mode, b.window) for b in banks]) as batch:
        d_in = [torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda() for x in xs]
        accs = [torch.zeros(batch.out_floats(i), dtype=torch.float32, device="cuda") for i in range(len(banks))]
        ns = [b.nspectra for b in banks]
        flags = batch.autotune(d_in, ns, accs, reps=2)
        assert len(flags) == len(banks)
        for i, f in enumerate(flags):  # the chosen plan form, split and launch shape are reported
            f2, shape = batch.bank_tuning(i)
            assert f2 == f and shape["blocks_a"] >= 0 and shape["blocks_b"] >= 0
            n2, cols = batch.bank_shape(i)
            print(f"\nbank {banks[i].nchan}: flags {f} col_len {n2} tile_cols {cols} {shape}")
        for rep in range(3):   # capture, replay, replay
            for a in accs:
                a.zero_()
            batch.execute(d_in, ns, accs)
            torch.cuda.synchronize()
            for b, a, o in zip(banks, accs, refs):
                assert_close(a.cpu().numpy().astype(np.float64).reshape(o.shape), o, what=f"batch {b.nchan} rep {rep}")
        accs2 = [torch.zeros_like(a) for a in accs]   # new pointers: re-capture
        batch.execute(d_in, ns, accs2)
        torch.cuda.synchronize()
        for a, a2 in zip(accs, accs2):
            assert torch.equal(a, a2)


@pytest.mark.parametrize("cfg,shapes", [
    ((32768, 8, 2, PFB, WIN_HANN, 21), [(8, 0), (16, 0), (32, 0), (64, 0), (16, 16), (16, 64)]),
    ((65536, 1, 2, DIRECT, WIN_RECT, 7), [(16, 0), (64, 0), (128, 0), (32, 64), (32, 128)]),
    ((8192, 3, 1, PFB, WIN_HAMMING, 9), [(2, 0), (8, 0), (4, 32), (4, 256)]),
], ids=["pfb32768", "direct65536", "single8192"])
def test_shaped_plans_match_oracle(oracle_mod, cfg, shapes):
    """Other four-step splits and kernel-A tile widths (the autotuner's
    candidates) give the oracle's spectrum; shapes the kernels cannot hold
    are refused."""
    from paper_1411_0436_gb300 import vspec
    n, p, npol, mode, win, s = cfg
    bank = Bank(n, p, npol, mode, win, s, rho=0.3 if npol == 2 else 0.0, tones=(Tone(30.0, n * 0.13 + 0.3, (0,)),))
    x = workloads.generate(bank, 61 + n)
    o = run_oracle(oracle_mod, bank, x)
    d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
    for n2, cols in shapes:
        with vspec.Plan(n, p, npol, mode, win, col_len=n2, tile_cols=cols) as plan:
            got_n2, got_cols = plan.shape()
            assert got_n2 == n2 and (cols == 0 or got_cols == cols), (plan.describe(), n2, cols)
            acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
            plan.execute(d_in, s, acc)
            torch.cuda.synchronize()
            g = acc.cpu().numpy().astype(np.float64)
        assert_close(g.reshape(n, 4) if npol == 2 else g, o, what=f"{cfg} shape {n2, cols}")
    for n2, cols in [(n, 0), (3, 0), (0, 3), (16, 1 << 14)]:
        with pytest.raises(vspec.VspecError) as e:
            vspec.Plan(n, p, npol, mode, win, col_len=n2, tile_cols=cols)
        assert e.value.status in (vspec.ERR_UNSUPPORTED, vspec.ERR_INVALID_ARG)


def test_trim_scratch_keeps_results(oracle_mod):
    """A plan whose chunk is set to its call length and whose scratch is
    trimmed holds less memory and gives the same spectrum."""
    from paper_1411_0436_gb300.vspec import Plan
    bank = Bank(131072, 8, 2, PFB, WIN_HANN, 37, rho=0.3)
    x = workloads.generate(bank, 808)
    o = run_oracle(oracle_mod, bank, x)
    d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
    with Plan(bank.nchan, 8, 2, PFB, WIN_HANN) as plan:
        before, _ = plan.info()
        plan.tune(chunk_spectra=bank.nspectra)
        plan.trim_scratch()
        after, _ = plan.info()
        assert after < before and before - after >= (2048 - 37) * 131072 * 16
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        plan.execute(d_in, bank.nspectra, acc)
        torch.cuda.synchronize()
        assert_close(acc.cpu().numpy().astype(np.float64).reshape(-1, 4), o, what="trimmed scratch")
        plan.tune(chunk_spectra=64)  # grows again
        assert plan.info()[0] > after


def test_plans_of_different_sizes_coexist():
    """A plan keeps working after another plan of the same kernels but smaller
    shared-memory needs was created (the kernels' shared-memory cap is shared)."""
    big = Bank(262144, 8, 2, PFB, WIN_HANN, 2)
    small = Bank(4096, 8, 2, PFB, WIN_HANN, 3)
    from paper_1411_0436_gb300.vspec import PLAN_TWO_KERNEL, Plan
    xb = workloads.generate(big, 1)
    xs = workloads.generate(small, 2)
    with Plan(big.nchan, 8, 2, PFB, WIN_HANN) as pb:
        with Plan(small.nchan, 8, 2, PFB, WIN_HANN, PLAN_TWO_KERNEL) as ps:
            db = torch.from_numpy(xb.view(np.uint8).reshape(-1)).cuda()
            ds = torch.from_numpy(xs.view(np.uint8).reshape(-1)).cuda()
            ab = torch.zeros(pb.out_floats, device="cuda")
            as_ = torch.zeros(ps.out_floats, device="cuda")
            ps.execute(ds, small.nspectra, as_)
            pb.execute(db, big.nspectra, ab)
            torch.cuda.synchronize()
            assert torch.isfinite(ab).all() and ab.abs().sum() > 0


@pytest.mark.parametrize("cfg", [(4096, 8, 2, PFB, WIN_HANN, 21, 8), (16384, 1, 2, DIRECT, WIN_RECT, 9, 8),
                                 (2048, 8, 1, PFB, WIN_HANN, 13, 8), (65536, 8, 2, PFB, WIN_HANN, 3, 8),
                                 (1024, 4, 2, PFB, WIN_HAMMING, 40, 3),
                                 # kernel A reading each band in place: PFB and direct register-column
                                 # forms, several 32 MiB chunks with a ragged last one
                                 (65536, 8, 2, PFB, WIN_HANN, 70, 4), (131072, 5, 2, PFB, WIN_HAMMING, 37, 8),
                                 (524288, 1, 2, DIRECT, WIN_RECT, 19, 2), (65536, 1, 2, DIRECT, WIN_HANN, 45, 8)])
def test_subband_mode_matches_oracle(oracle_mod, cfg):
    """Eight-sub-band modes (16 FFTs in parallel): input [time][sub][pol][re, im],
    output [sub][channel]; each sub-band equals the oracle on its own samples."""
    from paper_1411_0436_gb300.vspec import Plan
    n, p, npol, mode, win, s, nsub = cfg
    bank = Bank(n, p, npol, mode, win, s)
    xs = [workloads.generate(bank, 900 + 31 * b) for b in range(nsub)]
    x = np.ascontiguousarray(np.stack(xs, axis=1))          # [time][sub][pol][2]
    with Plan(n, p, npol, mode, win, nsub=nsub) as plan:
        assert x.nbytes == plan.input_bytes(s)
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        plan.execute(torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda(), s, acc)
        torch.cuda.synchronize()
        got = acc.cpu().numpy().astype(np.float64).reshape(nsub, -1)
    for b in range(nsub):
        o = run_oracle(oracle_mod, bank, np.ascontiguousarray(x[:, b]))
        assert_close(got[b].reshape(o.shape), o, what=f"{cfg} sub-band {b}")


@pytest.mark.parametrize("cfg", [(16384, 8, 2, PFB, WIN_HANN, 70, 3), (16384, 1, 2, DIRECT, WIN_HANN, 50, 5)])
def test_subband_in_place_band_by_band_matches_oracle(oracle_mod, cfg):
    """Two-kernel sub-band plans with short columns (no tiled fold): kernel A
    reads each band in place, one band after another over 32 MiB chunks."""
    from paper_1411_0436_gb300.vspec import PLAN_TWO_KERNEL, Plan
    n, p, npol, mode, win, s, nsub = cfg
    bank = Bank(n, p, npol, mode, win, s, rho=0.3, tones=(Tone(20.0, n * 0.3 + 0.2, (0,)),))
    x = np.ascontiguousarray(np.stack([workloads.generate(bank, 300 + 7 * b) for b in range(nsub)], axis=1))
    with Plan(n, p, npol, mode, win, PLAN_TWO_KERNEL, nsub=nsub) as plan:
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        plan.execute(torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda(), s, acc)
        torch.cuda.synchronize()
        got = acc.cpu().numpy().astype(np.float64).reshape(nsub, -1)
    for b in range(nsub):
        o = run_oracle(oracle_mod, bank, np.ascontiguousarray(x[:, b]))
        assert_close(got[b].reshape(o.shape), o, what=f"{cfg} band {b}")


@pytest.mark.parametrize("cfg", [(4096, 8, 2, PFB, WIN_HANN, 11), (32768, 8, 2, PFB, WIN_HANN, 30),
                                 (131072, 8, 2, PFB, WIN_HANN, 3), (524288, 1, 2, DIRECT, WIN_RECT, 2),
                                 (65536, 1, 2, DIRECT, WIN_RECT, 5),
                                 # tensor-core column DFTs: 16-, 32- and 64-point columns, ragged
                                 # batches, leading zero taps, windows
                                 (32768, 5, 2, PFB, WIN_RECT, 13), (65536, 8, 2, PFB, WIN_HANN, 21),
                                 (65536, 7, 2, PFB, WIN_HAMMING, 4), (131072, 8, 2, PFB, WIN_HANN, 37),
                                 (131072, 6, 2, PFB, WIN_HANN, 1)])
def test_tensor_core_plan_matches_oracle(oracle_mod, cfg):
    """First row pass on the tensor cores (bf16 hi/lo): within the tensor-core
    tolerance of the oracle."""
    from parity_util import ATOL_TC, metrics
    from paper_1411_0436_gb300.vspec import PLAN_TENSOR, Plan
    n, p, npol, mode, win, s = cfg
    bank = Bank(n, p, npol, mode, win, s, rho=0.3, tones=(Tone(40.0, n * 0.2 + 0.37, (0, 1)),))
    x = workloads.generate(bank, 321 + n)
    o = run_oracle(oracle_mod, bank, x)
    g = run_gpu(bank, x, flags=PLAN_TENSOR)
    m = assert_close(g, o, atol=ATOL_TC, what=f"{cfg} tensor")
    print(f"\n{cfg}: normalised max error {m['pure']:.3e} (fp32 path: "
          f"{metrics(run_gpu(bank, x), o)['pure']:.3e})")
    with Plan(n, p, npol, mode, win, PLAN_TENSOR) as plan:
        plan.check()


@pytest.mark.parametrize("cfg", [(32768, 8, 2, PFB, WIN_HANN, 30), (32768, 5, 2, PFB, WIN_RECT, 13),
                                 (65536, 8, 2, PFB, WIN_HANN, 21), (65536, 3, 2, PFB, WIN_HANN, 130),
                                 (131072, 8, 2, PFB, WIN_HANN, 37), (131072, 6, 2, PFB, WIN_HAMMING, 1),
                                 (32768, 1, 2, DIRECT, WIN_RECT, 300), (65536, 1, 2, DIRECT, WIN_RECT, 5),
                                 (131072, 1, 2, DIRECT, WIN_HANN, 7)],
                         ids=lambda c: f"N{c[0]}_P{c[1]}_m{c[3]}_w{c[4]}_S{c[5]}")
def test_int8_tensor_plan_matches_oracle(oracle_mod, cfg):
    """Pre-filter and column DFT as one tensor-core product on the int8
    input (128-spectrum blocks with ragged ends, fewer taps than the frame
    operand holds, windows, direct mode): within the tensor-core tolerance;
    the compensated form too."""
    from parity_util import ATOL_TC, metrics
    from paper_1411_0436_gb300.vspec import PLAN_KAHAN, PLAN_TENSOR_INT8, Plan
    n, p, npol, mode, win, s = cfg
    bank = Bank(n, p, npol, mode, win, s, rho=0.3, tones=(Tone(40.0, n * 0.2 + 0.37, (0, 1)),))
    x = workloads.generate(bank, 321 + n)
    o = run_oracle(oracle_mod, bank, x)
    m = assert_close(run_gpu(bank, x, flags=PLAN_TENSOR_INT8), o, atol=ATOL_TC, what=f"{cfg} int8 tensor")
    assert_close(run_gpu(bank, x, flags=PLAN_TENSOR_INT8 | PLAN_KAHAN), o, atol=ATOL_TC, what=f"{cfg} int8+kahan")
    print(f"\n{cfg}: normalised max error {m['pure']:.3e} (fp32 path: "
          f"{metrics(run_gpu(bank, x), o)['pure']:.3e})")
    with Plan(n, p, npol, mode, win, PLAN_TENSOR_INT8) as plan:
        assert "A=tensor-int8" in plan.describe()
        plan.check()


def test_int8_tensor_plan_rejects_other_sizes():
    from paper_1411_0436_gb300 import vspec
    for args in [(16384, 8, 2, PFB, WIN_HANN), (262144, 8, 2, PFB, WIN_HANN), (32768, 8, 1, PFB, WIN_HANN),
                 (32768, 12, 2, PFB, WIN_HANN)]:
        with pytest.raises(vspec.VspecError) as e:
            vspec.Plan(*args, flags=vspec.PLAN_TENSOR_INT8)
        assert e.value.status == vspec.ERR_UNSUPPORTED


def test_tensor_core_plan_rejects_other_sizes():
    from paper_1411_0436_gb300 import vspec
    for args in [(1024, 8, 2, PFB, WIN_HANN), (512, 1, 2, DIRECT, WIN_RECT), (32768, 8, 1, PFB, WIN_HANN)]:
        with pytest.raises(vspec.VspecError) as e:
            vspec.Plan(*args, flags=vspec.PLAN_TENSOR)
        assert e.value.status == vspec.ERR_UNSUPPORTED


@pytest.mark.parametrize("cfg", [(32768, 8, 2, PFB, WIN_HANN, 67), (4096, 1, 1, DIRECT, WIN_RECT, 40),
                                 (131072, 8, 2, PFB, WIN_HANN, 5), (1024, 8, 2, PFB, WIN_HANN, 500),
                                 (512, 1, 1, DIRECT, WIN_RECT, 700)])
def test_compensated_accumulation_matches_oracle(oracle_mod, cfg):
    """Kahan accumulation (alone and with the tensor-core pass) stays within
    the tolerances; dump clears the compensation with the accumulator."""
    from parity_util import ATOL_TC, metrics
    from paper_1411_0436_gb300.vspec import PLAN_KAHAN, PLAN_TENSOR, Plan
    n, p, npol, mode, win, s = cfg
    bank = Bank(n, p, npol, mode, win, s, rho=0.3 if npol == 2 else 0.0,
                tones=(Tone(50.0, n * 0.1 + 0.25, (0,)),))
    x = workloads.generate(bank, 4000 + n)
    o = run_oracle(oracle_mod, bank, x)
    mk = assert_close(run_gpu(bank, x, flags=PLAN_KAHAN), o, what=f"{cfg} kahan")
    mp = metrics(run_gpu(bank, x, flags=1), o)
    print(f"\n{cfg}: normalised max error plain {mp['pure']:.3e}, compensated {mk['pure']:.3e}")
    if npol == 2 and 2048 <= n <= 524288:  # the tensor-core pass needs 2048-point rows
        assert_close(run_gpu(bank, x, flags=PLAN_KAHAN | PLAN_TENSOR), o, atol=ATOL_TC,
                     what=f"{cfg} kahan+tensor")
    with Plan(n, p, npol, mode, win, PLAN_KAHAN) as plan:  # twice, dump in between
        d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        plan.execute(d_in, s, acc)
        plan.dump(acc)
        plan.execute(d_in, s, acc)
        torch.cuda.synchronize()
        assert_close(acc.cpu().numpy().astype(np.float64).reshape(o.shape), o, what=f"{cfg} after dump")


@pytest.mark.parametrize("cfg", [(65536, 8, 2, PFB, WIN_HANN, 37), (8192, 3, 1, PFB, WIN_HAMMING, 45),
                                 (262144, 1, 2, DIRECT, WIN_RECT, 9), (1024, 8, 2, PFB, WIN_HANN, 300),
                                 (2048, 5, 1, PFB, WIN_HAMMING, 61)],
                         ids=lambda c: f"N{c[0]}_P{c[1]}_pol{c[2]}_S{c[5]}")
def test_launch_shapes_match_oracle(oracle_mod, cfg):
    """Every launch shape of the two-kernel path (chunk length, CTAs per
    kernel-A and kernel-B launch, including one-spectrum chunks, a single CTA,
    CTAs that each hold a few items of several tiles, and the largest tuned
    launch) gives the oracle's spectrum."""
    from paper_1411_0436_gb300.vspec import Plan
    n, p, npol, mode, win, s = cfg
    bank = Bank(n, p, npol, mode, win, s, sigma=20.0, rho=0.3 if npol == 2 else 0.0,
                tones=(Tone(25.0, n * 0.3 + 0.4, (0, 1)),))
    x = workloads.generate(bank, 77 + n)
    o = run_oracle(oracle_mod, bank, x)
    d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8).reshape(-1)).cuda()
    with Plan(n, p, npol, mode, win) as plan:
        cur, lim = plan.get_tuning()
        assert 1 <= cur["chunk_spectra"] <= lim["chunk_spectra"]
        assert cur["blocks_a"] == cur["blocks_b"] == 0 and lim["blocks_a"] > 0 and lim["blocks_b"] > 0
        shapes = [(1, 0, 0), (1, 1, 1), (min(5, lim["chunk_spectra"]), 3, 2), (2, 7, 13),
                  (lim["chunk_spectra"], 7, lim["blocks_b"]), (lim["chunk_spectra"], 0, 1),
                  (cur["chunk_spectra"], lim["blocks_a"], 0)]
        for chunk, ba, bb in shapes:
            plan.tune(chunk_spectra=chunk, blocks_a=ba, blocks_b=bb)
            acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
            plan.execute(d_in, s, acc)
            torch.cuda.synchronize()
            g = acc.cpu().numpy().astype(np.float64)
            assert_close(g.reshape(n, 4) if npol == 2 else g, o, what=f"{cfg} shape {chunk, ba, bb}")


def test_tuning_limits():
    from paper_1411_0436_gb300.vspec import NEVER, Plan, VspecError
    import paper_1411_0436_gb300.vspec as V

    def rejected(plan, **bad):
        before = plan.get_tuning()[0]
        with pytest.raises(VspecError) as e:
            plan.tune(**bad)
        assert e.value.status == V.ERR_INVALID_ARG
        assert plan.get_tuning()[0] == before  # a rejected shape changes nothing

    with Plan(65536, 8, 2, PFB, WIN_HANN) as plan:  # two-kernel plan
        cur, lim = plan.get_tuning()
        assert cur["two_kernel_from"] == 0 and lim["assist_permille"] == 0
        for bad in [dict(chunk_spectra=0), dict(chunk_spectra=lim["chunk_spectra"] + 1), dict(blocks_a=-1),
                    dict(blocks_a=lim["blocks_a"] + 1), dict(blocks_b=-1), dict(blocks_b=lim["blocks_b"] + 1),
                    dict(assist_permille=5), dict(two_kernel_from=7)]:
            rejected(plan, **bad)
    with Plan(32768, 8, 2, PFB, WIN_HANN) as plan:  # fused plan owning a two-kernel plan
        cur, lim = plan.get_tuning()
        assert cur["chunk_spectra"] >= 1 and lim["two_kernel_from"] == NEVER
        assert 0 <= cur["assist_permille"] <= lim["assist_permille"] <= 1000
        for bad in [dict(chunk_spectra=0), dict(assist_permille=-1),
                    dict(assist_permille=lim["assist_permille"] + 1), dict(two_kernel_from=-1)]:
            rejected(plan, **bad)
        plan.tune(two_kernel_from=NEVER, assist_permille=0)
    with Plan(2048, 8, 2, PFB, WIN_HANN) as plan:  # fused, no two-kernel plan
        cur, lim = plan.get_tuning()
        assert cur == {"chunk_spectra": 0, "blocks_a": 0, "blocks_b": 0, "assist_permille": 0,
                       "two_kernel_from": NEVER}
        rejected(plan, two_kernel_from=100)
        rejected(plan, chunk_spectra=4)


@pytest.mark.parametrize("cfg", [(32768, 8, 2, PFB, WIN_HANN, 150), (8192, 1, 2, DIRECT, WIN_RECT, 900)],
                         ids=lambda c: f"N{c[0]}_m{c[3]}_S{c[5]}")
def test_fused_plan_switches_to_two_kernel_path(oracle_mod, cfg):
    """A fused plan runs a call wholly on its two-kernel plan from
    two_kernel_from spectra on, and on the cluster kernel below; both give
    the oracle's spectrum and the profiling records show which path ran."""
    from paper_1411_0436_gb300.vspec import NEVER, Plan
    n, p, npol, mode, win, s = cfg
    bank = Bank(n, p, npol, mode, win, s, sigma=20.0, rho=0.3, tones=(Tone(25.0, n * 0.3 + 0.4, (0, 1)),))
    x = workloads.generate(bank, 55 + n)
    o = run_oracle(oracle_mod, bank, x)
    d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8).reshape(-1)).cuda()
    with Plan(n, p, npol, mode, win) as plan:
        for threshold, two_kernel in ((s, True), (s + 1, False), (0, True), (NEVER, False)):
            plan.tune(two_kernel_from=threshold, assist_permille=0)
            plan.set_profiling(True)
            acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
            plan.execute(d_in, s, acc)
            torch.cuda.synchronize()
            stats = {r[0]: r for r in plan.kernel_stats()}
            plan.set_profiling(False)
            assert_close(acc.cpu().numpy().astype(np.float64).reshape(n, 4), o, what=f"{cfg} from {threshold}")
            assert (stats["fir_colfft"][2] == s) == two_kernel
            assert (stats["fused_channelize"][2] == s) == (not two_kernel)


@pytest.mark.parametrize("cfg", [(32768, 8, 2, PFB, WIN_HANN, 300), (32768, 1, 2, DIRECT, WIN_HAMMING, 233),
                                 (4096, 1, 2, DIRECT, WIN_RECT, 500),
                                 (2048, 8, 2, PFB, WIN_HAMMING, 150)],
                         ids=lambda c: f"N{c[0]}_P{c[1]}_m{c[3]}_S{c[5]}")
def test_fused_assist_shares_match_oracle(oracle_mod, cfg):
    """A fused plan splits the spectra between the cluster kernel and a
    concurrent two-kernel pass on the idle SMs; every split (none, the
    default, half, the maximum) gives the oracle's spectrum, and the
    profiling records cover both paths' kernels."""
    from paper_1411_0436_gb300.vspec import NEVER, Plan
    n, p, npol, mode, win, s = cfg
    bank = Bank(n, p, npol, mode, win, s, sigma=20.0, rho=0.3, tones=(Tone(25.0, n * 0.3 + 0.4, (0, 1)),))
    x = workloads.generate(bank, 99 + n)
    o = run_oracle(oracle_mod, bank, x)
    d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8).reshape(-1)).cuda()
    with Plan(n, p, npol, mode, win) as plan:
        cur, lim = plan.get_tuning()
        for share in sorted({0, cur["assist_permille"], min(500, lim["assist_permille"]), lim["assist_permille"]}):
            plan.tune(assist_permille=share, two_kernel_from=NEVER)
            plan.set_profiling(True)
            acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
            plan.execute(d_in, s, acc)
            torch.cuda.synchronize()
            stats = {r[0]: r for r in plan.kernel_stats()}
            plan.set_profiling(False)
            assert_close(acc.cpu().numpy().astype(np.float64).reshape(n, 4), o, what=f"{cfg} assist {share}")
            sa = stats["fir_colfft"][2]  # spectra the assist channelized
            assert sa in (0, s * share // 1000) and (share > 0 or sa == 0)
            assert stats["fused_channelize"][2] + sa == s


@pytest.mark.parametrize("cfg,expect", [
    ((32768, 8, 2, PFB, WIN_HANN, 0), ("fused K=16", "A=colreg", "N2=16", "B=row2048")),   # c2
    ((524288, 1, 2, DIRECT, WIN_RECT, 0), ("two-kernel", "A=coldir", "N2=256", "B=row2048")),  # c3
    ((131072, 8, 2, PFB, WIN_HANN, 0), ("A=colreg", "N2=64", "C=8", "B=row2048")),         # c4
    ((262144, 8, 2, PFB, WIN_HANN, 0), ("A=colreg", "N2=128", "C=4")),
    ((524288, 8, 2, PFB, WIN_HANN, 0), ("A=colreg", "N1=4096", "B=row4096")),
    ((1 << 20, 8, 2, PFB, WIN_HANN, 0), ("A=gather", "N1=2048")),
    ((1024, 8, 1, PFB, WIN_HANN, 0), ("A=none", "fir-in-B", "B=general")),              # c1
    ((65536, 4, 1, PFB, WIN_HANN, 0), ("A=general",)),
])
def test_plans_choose_the_intended_kernels(cfg, expect):
    """The fast kernel forms are chosen where they apply (a silent fallback to
    the general kernels would still match the oracle, only slower)."""
    from paper_1411_0436_gb300.vspec import Plan
    n, p, npol, mode, win, _ = cfg
    with Plan(n, p, npol, mode, win) as plan:
        d = plan.describe()
    for word in expect:
        assert word in d, (cfg, d)
