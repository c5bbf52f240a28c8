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


def group_spans(tiles, sc, n, G):
    """Kernel A's grouped split: n // G groups take block_span shares of the
    tiles // G super-tiles; member r of a group the r-th tile of each."""
    ng = n // G
    T = (tiles // G) * sc
    for k in range(n):
        g, r = k // G, k % G
        if g >= ng:
            continue
        lo, hi = T * g // ng, T * (g + 1) // ng
        f = lo
        while f < hi:
            base = f // sc * sc
            x = (f // sc) * G + r
            s_end = min(hi, base + sc) - base
            yield k, x, f - base, s_end
            f = base + s_end


def host_grid(n_a, tiles, sc, G):
    """The host's kernel-A grid: at most one block per item, a whole number of groups."""
    ga = min(n_a, tiles * sc)
    return max(G, ga // G * G)


@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_tile_groups_cover_every_item_once(G):
    for tiles in (G, 2 * G, 16, 64, 256):
        if tiles % G:
            continue
        for sc in (1, 2, 5, 33, 512):
            for n_a in (1, 3, 7, 152, 304):
                n = host_grid(n_a, tiles, sc, G)
                assert n % G == 0
                seen = [0] * (tiles * sc)
                for k, x, s_beg, s_end in group_spans(tiles, sc, n, G):
                    assert x % G == k % G  # a member keeps its lane of every super-tile
                    for s in range(s_beg, s_end):
                        seen[x * sc + s] += 1
                assert seen == [1] * (tiles * sc), (tiles, sc, n, G)


def test_group_members_walk_the_same_spectra():
    # the members of a group read adjacent tiles of the same frames in step
    tiles, sc, n, G = 256, 512, 152, 4
    by_block = {}
    for k, x, s_beg, s_end in group_spans(tiles, sc, n, G):
        by_block.setdefault(k, []).append((x // G, s_beg, s_end))
    for g in range(n // G):
        runs = [by_block[g * G + r] for r in range(G)]
        assert all(run == runs[0] for run in runs)
