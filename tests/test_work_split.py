"""The balanced split of a two-kernel launch's work (tile x spectrum items,
tile-major; block k of n takes items [k T / n, (k+1) T / n)) and the partial-
sum slot each block uses for a tile (its rank among the blocks that meet the
tile). The kernels compute both in integer arithmetic; the plan allocates
n // tiles + 2 slots. This checks, over every small shape, that the rank
formula names the block holding the tile's first item and stays below that
bound, and that the segments cover every item exactly once."""
import itertools

import pytest


def spans(tiles, sc, n):
    T = tiles * sc
    for k in range(n):
        lo, hi = T * k // n, T * (k + 1) // n
        f = lo
        while f < hi:
            x = f // sc
            base = x * sc
            s_end = min(hi, base + sc) - base
            k_lo = ((x * sc + 1) * n - 1) // T
            yield k, x, f - base, s_end, k_lo
            f = base + s_end


@pytest.mark.parametrize("tiles", [1, 2, 3, 7, 16, 64])
def test_slots_cover_and_stay_in_bound(tiles):
    T_shapes = [(sc, n) for sc in (1, 2, 5, 16, 33) for n in (1, 3, 7, 64, 152, 304, 1000)]
    for sc, n in T_shapes:
        T = tiles * sc
        seen = [0] * T
        users = {}
        for k, x, s_beg, s_end, k_lo in spans(tiles, sc, n):
            assert T * k_lo // n <= x * sc < T * (k_lo + 1) // n
            slot = k - k_lo
            assert 0 <= slot < n // tiles + 2
            # no two blocks write the same (tile, slot) in one launch
            assert (x, slot) not in users
            users[(x, slot)] = k
            for s in range(s_beg, s_end):
                seen[x * sc + s] += 1
        assert seen == [1] * T, (tiles, sc, n)
