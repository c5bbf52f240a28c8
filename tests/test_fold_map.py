"""Index map of the tiled fold for 2048-point rows (reduce2048_kernel),
restated on the CPU: the rows pass radices 16, 16, 8 in decimation-in-
frequency order, so row position posB holds output k1 by digit reversal.
Every block's read side (slot row, position) and write side (channel) must
name the same channel, and the blocks together must cover every channel of
the transform exactly once."""
import pytest


def digit_reverse(length, radices):
    """k held at each position after in-place DIF passes of these radices."""
    out = []
    for pos in range(length):
        rem, lb, k, scale = pos, length, 0, 1
        for r in radices:
            m = lb // r
            q = rem // m
            rem -= q * m
            k += q * scale
            scale *= r
            lb = m
        out.append(k)
    return out


def blocks(n2, pb):
    """(k2, posB) read and channel written for every tile element, per block."""
    nk, q2g = n2 // 16, pb // 8
    for b in range(nk * 16 * (128 // pb)):
        k2_0 = 16 * (b % nk)
        q1, g = (b // nk) % 16, b // (nk * 16)
        p0 = 128 * q1 + pb * g
        reads = {}
        for e in range(16 * pb):
            r, j = e // pb, e % pb
            reads[(r, j)] = (k2_0 + r, p0 + j)
        writes = {}
        for e in range(16 * pb):
            r, j = e & 15, e >> 4
            k1 = q1 + 16 * (q2g * g + (j >> 3)) + 256 * (j & 7)
            writes[(r, j)] = k1 * n2 + k2_0 + r
        yield reads, writes


def test_row_positions_follow_the_digit_reversal():
    kb = digit_reverse(2048, (16, 16, 8))
    for pos in range(2048):
        q1, q2, q3 = pos // 128, (pos // 8) % 16, pos % 8
        assert kb[pos] == q1 + 16 * q2 + 256 * q3


@pytest.mark.parametrize("n2,pb", [(16, 8), (32, 8), (64, 32), (256, 32), (512, 32)])
def test_reads_and_writes_name_the_same_channel_once(n2, pb):
    kb = digit_reverse(2048, (16, 16, 8))
    seen = [0] * (n2 * 2048)
    for reads, writes in blocks(n2, pb):
        for key, (k2, posb) in reads.items():
            k = writes[key]
            assert k == k2 + n2 * kb[posb]
            seen[k] += 1
    assert seen == [1] * (n2 * 2048)
