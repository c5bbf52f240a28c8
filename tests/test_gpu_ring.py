"""The persistent ring form (VSPEC_PLAN_RING) against the FP64 oracle.

One cooperative launch per call runs kernel-A and kernel-B tickets in
dependency order, with the four-step intermediate in a ring of a few slots.
These tests cover ragged last slots (odd spectrum counts, half-empty kernel-B
groups), every column length the ring holds, small rings that force the
waits (one slot, lookahead 1), calls long enough to need two launches,
sub-band plans, bitwise reproducibility, the full c2 and c4 dumps, and the
failure path of a wait that gives up (injected from the host: the counter it
waits for starts one short, so nothing faults).
"""
import numpy as np
import pytest

from parity_util import assert_close, metrics
from paper_1411_0436_gb300 import workloads
from paper_1411_0436_gb300.workloads import PFB, WIN_HAMMING, WIN_HANN, Bank, Tone
from test_gpu_parity import run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def ring_run(bank: Bank, x: np.ndarray, shape=None, repeat: int = 1, nsub: int = 1) -> np.ndarray:
    from paper_1411_0436_gb300.vspec import PLAN_RING, Plan
    with Plan(bank.nchan, bank.ntaps, bank.npol, bank.mode, bank.window, PLAN_RING, nsub=nsub) as plan:
        if shape:
            plan.set_ring(**shape)
        d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.uint8).reshape(-1)).cuda()
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        for _ in range(repeat):
            plan.execute(d_in, bank.nspectra, acc)
        torch.cuda.synchronize()
        plan.check()
        out = acc.cpu().numpy().astype(np.float64)
    if nsub > 1:
        return out.reshape(nsub, bank.nchan, 4)
    return out.reshape(bank.nchan, 4)


def bank_of(n, s, taps=8, window=WIN_HANN):
    return Bank(n, taps, 2, PFB, window, s, rho=0.3, tones=(Tone(30.0, n * 0.37 + 0.25, (0,)),
                                                            Tone(9.0, n * 0.61 + 0.5, (0, 1))))


# nchan, spectra, ring shape (None: the plan's default)
CASES = [
    (4096, 1100, None),                                   # N2 = 2: 512-spectrum slots, 32 tickets per row
    (8192, 301, None),                                    # N2 = 4
    (16384, 300, None),                                   # N2 = 8, ragged last slot
    (32768, 201, None),                                   # N2 = 16, odd: a half-empty group
    (65536, 70, None),                                    # N2 = 32
    (131072, 45, None),                                   # N2 = 64 (the headline's column length)
    (262144, 19, None),                                   # N2 = 128
    (131072, 40, dict(slot_spectra=4, ring_slots=2, lookahead=1, row_parts=1)),
    (131072, 23, dict(slot_spectra=2, ring_slots=1, lookahead=1, row_parts=1)),  # every wait taken
    (32768, 130, dict(slot_spectra=16, ring_slots=4, lookahead=3, row_parts=8)),
    (16384, 97, dict(slot_spectra=32, ring_slots=16, lookahead=15, row_parts=1)),
]


@pytest.mark.parametrize("n,s,shape", CASES, ids=[f"N{c[0]}_S{c[1]}_{'default' if c[2] is None else 'shaped'}"
                                                 for c in CASES])
def test_ring_matches_oracle(oracle_mod, n, s, shape):
    bank = bank_of(n, s)
    x = workloads.generate(bank, 4200 + n + s)
    g = ring_run(bank, x, shape)
    m = assert_close(g, run_oracle(oracle_mod, bank, x), what=f"ring N={n} S={s} {shape}")
    print(f"\nring N={n} spectra={s} {shape}: max err / RMS {m['pure']:.2e}, tolerance use {m['ratio']:.3f}")


def test_ring_other_taps_and_window(oracle_mod):
    bank = bank_of(32768, 77, taps=5, window=WIN_HAMMING)
    x = workloads.generate(bank, 99)
    assert_close(ring_run(bank, x), run_oracle(oracle_mod, bank, x), what="ring 5 taps Hamming")


def test_ring_two_launches(oracle_mod):
    """More slots than one launch's done counters hold (4096): two launches,
    the second continuing the first's partial-sum sets."""
    bank = bank_of(4096, 8195)
    x = workloads.generate(bank, 7)
    g = ring_run(bank, x, dict(slot_spectra=2, ring_slots=3, lookahead=2, row_parts=1))
    assert_close(g, run_oracle(oracle_mod, bank, x), what="ring over two launches")


def test_ring_accumulates_and_is_reproducible(oracle_mod):
    bank = bank_of(131072, 37)
    x = workloads.generate(bank, 11)
    a = ring_run(bank, x, repeat=2)
    b = ring_run(bank, x, repeat=2)
    assert np.array_equal(a, b), "ring results differ between identical runs"
    assert_close(a, 2.0 * run_oracle(oracle_mod, bank, x), what="ring, two calls into one accumulator")


def test_ring_subbands(oracle_mod):
    """Sub-band input [time][sub][pol][re, im]: each sub-band equals the oracle on its own samples."""
    bank = bank_of(16384, 40)
    xs = [workloads.generate(bank, 600 + 13 * b) for b in range(2)]
    x = np.ascontiguousarray(np.stack(xs, axis=1))
    g = ring_run(bank, x, nsub=2)
    for b in range(2):
        assert_close(g[b], run_oracle(oracle_mod, bank, np.ascontiguousarray(x[:, b])), what=f"ring sub-band {b}")


def test_ring_plan_properties():
    from paper_1411_0436_gb300.vspec import (ERR_INVALID_ARG, ERR_UNSUPPORTED, PLAN_RING, PLAN_KAHAN, Plan,
                                             VspecError, DIRECT, WIN_RECT)
    with Plan(131072, 8, 2, PFB, WIN_HANN, PLAN_RING) as plan:
        assert plan.ring() == dict(slot_spectra=16, ring_slots=3, lookahead=2, row_parts=1)
        scratch, passes = plan.info()
        assert passes == 1
        assert scratch < 160 << 20, scratch  # ring 96 MiB + sets 16 MiB + tables
        assert "ring S=16" in plan.describe()
        with pytest.raises(VspecError) as e:
            plan.set_tuning(1, 0, 0, 0, 0)
        assert e.value.status == ERR_UNSUPPORTED
        for bad in (dict(slot_spectra=3), dict(ring_slots=1, lookahead=2), dict(slot_spectra=16, row_parts=3),
                    dict(slot_spectra=128, row_parts=2)):
            with pytest.raises(VspecError) as e:
                plan.set_ring(**bad)
            assert e.value.status == ERR_INVALID_ARG, bad
        plan.set_ring(slot_spectra=8)
        assert plan.ring() == dict(slot_spectra=8, ring_slots=3, lookahead=2, row_parts=1)
    for args in ((524288, 1, 2, DIRECT, WIN_RECT, PLAN_RING), (131072, 8, 1, PFB, WIN_HANN, PLAN_RING),
                 (131072, 8, 2, PFB, WIN_HANN, PLAN_RING | PLAN_KAHAN), (1024, 8, 2, PFB, WIN_HANN, PLAN_RING)):
        with pytest.raises(VspecError) as e:
            Plan(*args)
        assert e.value.status == ERR_UNSUPPORTED, args
    with Plan(131072, 8, 2, PFB, WIN_HANN) as plan:
        with pytest.raises(VspecError) as e:
            plan.set_ring(slot_spectra=8)
        assert e.value.status == ERR_UNSUPPORTED


def test_ring_wait_that_gives_up_is_reported_and_plan_recovers(oracle_mod):
    from paper_1411_0436_gb300.vspec import ERR_DEVICE_TIMEOUT, PLAN_RING, Plan, VspecError, vspec_set_wait_limit
    bank = bank_of(131072, 50)
    x = workloads.generate(bank, 21)
    o = run_oracle(oracle_mod, bank, x)
    with Plan(bank.nchan, 8, 2, PFB, WIN_HANN, PLAN_RING) as plan:
        d_in = torch.from_numpy(x.view(np.uint8).reshape(-1)).cuda()
        acc = torch.zeros(plan.out_floats, dtype=torch.float32, device="cuda")
        vspec_set_wait_limit(20000)  # about 2 ms per wait
        try:
            plan.inject_stall(1)
            plan.execute(d_in, bank.nspectra, acc)
            torch.cuda.synchronize()
            with pytest.raises(VspecError) as e:
                plan.check()
            assert e.value.status == ERR_DEVICE_TIMEOUT
            plan.check()  # reported once
        finally:
            vspec_set_wait_limit(-1)
        acc.zero_()
        plan.execute(d_in, bank.nspectra, acc)
        torch.cuda.synchronize()
        plan.check()
        assert_close(acc.cpu().numpy().astype(np.float64).reshape(bank.nchan, 4), o, what="ring after a timeout")


@pytest.mark.slow
@pytest.mark.parametrize("name", ["c2", "c4"])
def test_ring_full_workload(oracle_mod, name):
    bank = workloads.CONFIGS[name][0]
    x = workloads.generate(bank, workloads.config_seed(name))
    o = run_oracle(oracle_mod, bank, x)
    m = assert_close(ring_run(bank, x), o, what=f"{name} ring")
    print(f"\n{name} ring: max err / RMS {m['pure']:.3e}, tolerance use {m['ratio']:.3f}")
