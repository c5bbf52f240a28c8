"""Index maps of the tensor-core column kernel (fir_coltc_kernel), restated
on the CPU for its three column lengths (N2 = 16, 32, 64; C = 512 / N2
columns per tile, 8 spectra per batch):

* the frame staging: each thread's fixed 16-byte copies land every
  (spectrum, point) of a batch exactly once, at the point's slot;
* the pre-filter's operand offsets: point (n2, c) of spectrum u and
  polarisation p goes to row 8 (2 (u C/8 + c/8) + p) + c mod 8, K = 2 n2,
  and each warp's 32 stores for one (u, p) hit 32 different banks;
* the epilogue: the .16x256b fragment a thread reads (rows r0 and r0 + 8 of
  its 16-lane half, columns 2 (lane mod 4) + 8 i) is the X and Y
  polarisation of one (spectrum, column, k2), and the 16 warps together
  write every scratch element of the batch exactly once.
"""
import pytest

PTS, SPB = 512, 8


def geometry(n2):
    c = PTS // n2
    k = 2 * n2
    return dict(C=c, CB=c // 8, K=k, NN=k, SBO=k * 16)


def pt_n2(t, g):
    return ((t >> 5) // g["CB"]) * 4 + ((t >> 3) & 3)


def pt_c(t, g):
    return ((t >> 5) % g["CB"]) * 8 + (t & 7)


def pt_index(n2, c, g):
    return ((n2 >> 2) * g["CB"] + (c >> 3)) * 32 + (n2 & 3) * 8 + (c & 7)


def off(r, k, g):
    """Byte offset of element (row r, k) in the K-major no-swizzle layout."""
    return (r >> 3) * g["SBO"] + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2


def row(u, pol, c, g):
    C = g["C"]
    return 8 * (2 * (u * (C // 8) + c // 8) + pol) + c % 8


@pytest.mark.parametrize("n2", [16, 32, 64])
def test_thread_order_is_a_permutation_of_the_tile(n2):
    g = geometry(n2)
    pts = {(pt_n2(t, g), pt_c(t, g)) for t in range(PTS)}
    assert pts == {(a, b) for a in range(n2) for b in range(g["C"])}
    assert all(pt_index(pt_n2(t, g), pt_c(t, g), g) == t for t in range(PTS))


@pytest.mark.parametrize("n2", [16, 32, 64])
@pytest.mark.parametrize("nbb", [1, 3, 4, 5, 8])
def test_staging_copies_cover_the_batch_once(n2, nbb):
    g = geometry(n2)
    per_row, per_frame = g["C"] // 4, PTS // 4
    seen = []
    for t in range(PTS):
        st_u, st_r = t // per_frame, t % per_frame
        st_n2, st_ch = st_r // per_row, st_r % per_row
        st_dst = st_u * PTS + pt_index(st_n2, st_ch * 4, g)
        for i in range(SPB // 4):
            u = st_u + 4 * i
            if u >= nbb:
                continue
            for j in range(4):  # the 4 words of the 16-byte copy
                c = st_ch * 4 + j
                assert st_dst + 4 * PTS * i + j == u * PTS + pt_index(st_n2, c, g)
                seen.append((u, st_n2, c))
    assert sorted(seen) == sorted((u, a, b) for u in range(nbb) for a in range(n2) for b in range(g["C"]))


@pytest.mark.parametrize("n2", [16, 32, 64])
def test_operand_rows_are_a_permutation_and_stores_are_conflict_free(n2):
    g = geometry(n2)
    C, SBO = g["C"], g["SBO"]
    rows = {row(u, p, c, g) for u in range(SPB) for p in range(2) for c in range(C)}
    assert rows == set(range(SPB * 2 * C))
    for w in range(PTS // 32):
        for u in range(SPB):
            for p in range(2):
                banks = set()
                for lane in range(32):
                    t = 32 * w + lane
                    n2_, c = pt_n2(t, g), pt_c(t, g)
                    o_y = off(16 * (c >> 3) + (c & 7), 2 * n2_, g)
                    o = o_y + 2 * u * (C // 8) * SBO + p * SBO
                    assert o == off(row(u, p, c, g), 2 * n2_, g)
                    banks.add((o // 4) % 32)
                assert len(banks) == 32


@pytest.mark.parametrize("n2", [16, 32, 64])
def test_epilogue_fragments_pair_the_polarisations(n2):
    g = geometry(n2)
    C, NN = g["C"], g["NN"]
    written = set()
    for warp in range(16):
        q, gi = warp & 3, warp >> 2
        mb, k0 = (32 * gi) // NN, ((32 * gi) % NN) // 2
        for h in range(2):
            pr = 8 * mb + 2 * q + h
            eu, ecb = pr // (C // 8), pr % (C // 8)
            for lane in range(32):
                ec = ecb * 8 + (lane >> 2)
                lane_x = 32 * q + 16 * h + (lane >> 2)  # fragment rows r0 and r0 + 8
                assert mb * 128 + lane_x == row(eu, 0, ec, g)
                assert mb * 128 + lane_x + 8 == row(eu, 1, ec, g)
                for r in range(4):
                    col = (32 * gi) % NN + 8 * r + 2 * (lane & 3)  # (re, im) of output col / 2
                    k2 = k0 + 4 * r + (lane & 3)
                    assert col // 2 == k2 and col % 2 == 0
                    key = (eu, ec, k2)
                    assert key not in written
                    written.add(key)
    assert len(written) == SPB * C * n2
