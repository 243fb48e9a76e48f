"""The rotate-and-select step of the cross-lane 32x32 bit transpose that
builds a mixed-key tile's table (transpose_lanes32 in csrc/tdes_mixed.cuh),
modelled on the host: lane i starts with row i of the matrix and must end
with column i.  Each step exchanges blocks of width w between lanes i and
i ^ w; the lane whose bit w is set rotates its partner's word left by
32 - w, the other by w, and keeps its own block under a per-lane mask.  The
model is compared with a plain transpose and with the two-branch form
(mask, shift and OR on each side) it replaced.  The kernels themselves are
covered by the mixed-key GPU parity tests."""
import random

M = 0xFFFFFFFF
HI = {16: 0xFFFF0000, 8: 0xFF00FF00, 4: 0xF0F0F0F0, 2: 0xCCCCCCCC, 1: 0xAAAAAAAA}


def rotl(y, s):
    s &= 31
    return ((y << s) | (y >> (32 - s))) & M if s else y


def rotate_select(rows):
    xs = list(rows)
    for w in (16, 8, 4, 2, 1):
        ys = [xs[lane ^ w] for lane in range(32)]
        nxt = []
        for lane, (x, y) in enumerate(zip(xs, ys)):
            upper = bool(lane & w)
            keep = HI[w] if upper else ~HI[w] & M
            r = rotl(y, 32 - w if upper else w)
            nxt.append((x & keep) | (r & ~keep & M))
        xs = nxt
    return xs


def two_branch(rows):
    xs = list(rows)
    for w in (16, 8, 4, 2, 1):
        hi = HI[w]
        ys = [xs[lane ^ w] for lane in range(32)]
        xs = [((x & hi) | ((y & hi) >> w)) if lane & w
              else ((x & ~hi & M) | (((y & ~hi & M) << w) & M))
              for lane, (x, y) in enumerate(zip(xs, ys))]
    return xs


def columns(rows):
    return [sum(((rows[i] >> c) & 1) << i for i in range(32)) for c in range(32)]


def test_rotate_select_is_a_transpose():
    rng = random.Random(3)
    cases = [[0] * 32, [M] * 32, [1 << i for i in range(32)], [M >> i for i in range(32)]]
    cases += [[rng.getrandbits(32) for _ in range(32)] for _ in range(300)]
    for rows in cases:
        want = columns(rows)
        assert rotate_select(rows) == want
        assert two_branch(rows) == want
        assert rotate_select(want) == rows  # a transpose is its own inverse
