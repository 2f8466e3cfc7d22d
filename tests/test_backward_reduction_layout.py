"""The render backward's warp reduction of a pair's gradient values (csrc/render.cu): host-side
model of the recursive halving, checked against the kernel's packed position -> slot tables.

The backward sums NV values per (warp, splat) event across the 32 lanes: at the level with lane
offset 16 each lane keeps positions [0, NV/2) or [NV/2, NV) (bit 16 clear / set) and adds its
partner's copy; levels 8, 4 and 2 halve the remaining values the same way (the upper half padded
with a zero when odd), and the last level sums each lane pair. The even lane of a pair then adds
its sum into the splat's 16-float accumulator at slot (kSlots >> 4 * position) & 15. These tests
read kSlots from the source, run the model on random integers, and check that every slot gets
exactly the warp sum of one position and that the slots are the accumulator layout the
preprocess backward reads: 0-1 mean, 2-4 Sigma', 5 opacity, 6 beta, 7 depth, 8-10 colour,
12-14 normal (without depth and normal: 0-6 and 8-10)."""
import os
import random
import re

import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2411_09156_gb300", "csrc", "render.cu")


def _tables():
    txt = open(SRC).read()
    m = re.search(r"kSlots\s*=\s*FULL\s*\?\s*(0x[0-9A-Fa-f]+)ull\s*:\s*(0x[0-9A-Fa-f]+)ull", txt)
    assert m, "packed slot tables not found in render.cu"
    nv = re.search(r"constexpr int NV = FULL \? (\d+) : (\d+);", txt)
    assert nv, "value counts not found in render.cu"
    return {True: (int(nv.group(1)), int(m.group(1), 16)), False: (int(nv.group(2)), int(m.group(2), 16))}


def _reduce_label(nv, lane):
    """Position a lane pair holds after the halvings, or -1 (padding), as the kernel computes it."""
    start, valid, n = 0, nv, nv
    d = 16
    while d >= 2:
        h = (n + 1) // 2
        if lane & d:
            start += h
            valid = valid - h if valid > h else 0
        else:
            valid = min(valid, h)
        n = h
        d >>= 1
    return start if valid > 0 else -1


def _warp_sums(vals, nv):
    """vals[lane][position] -> {position: sum}, through the kernel's sequence of halvings."""
    h1 = nv // 2
    g = []
    for lane in range(32):
        up, p = bool(lane & 16), lane ^ 16
        keep = [vals[lane][i + h1] if up else vals[lane][i] for i in range(h1)]
        recv = [vals[p][i] if (p & 16) else vals[p][i + h1] for i in range(h1)]
        g.append([k + r for k, r in zip(keep, recv)])
    n = h1
    for d in (8, 4, 2):
        h = (n + 1) // 2
        new = []
        for lane in range(32):
            up, p = bool(lane & d), lane ^ d
            row = []
            for i in range(h):
                rest_l = g[lane][h + i] if h + i < n else 0
                rest_p = g[p][h + i] if h + i < n else 0
                keep = rest_l if up else g[lane][i]
                send_p = g[p][i] if (p & d) else rest_p
                row.append(keep + send_p)
            new.append(row)
        g, n = new, h
    out = {}
    for lane in range(0, 32, 2):
        lab = _reduce_label(nv, lane)
        if lab >= 0:
            assert lab not in out
            out[lab] = g[lane][0] + g[lane + 1][0]
    return out


@pytest.mark.parametrize("full", [True, False])
def test_every_position_reaches_its_slot_with_the_warp_sum(full):
    nv, table = _tables()[full]
    rng = random.Random(7 + nv)
    vals = [[rng.randint(-10**6, 10**6) for _ in range(nv)] for _ in range(32)]
    sums = _warp_sums(vals, nv)
    assert sorted(sums) == list(range(nv))  # every position ends in exactly one lane pair
    for pos in range(nv):
        assert sums[pos] == sum(v[pos] for v in vals)
    slots = [(table >> (4 * pos)) & 15 for pos in range(nv)]
    assert len(set(slots)) == nv  # one slot per position
    want = set(range(11)) | {12, 13, 14} if full else set(range(7)) | {8, 9, 10}
    assert set(slots) == want
    assert table >> (4 * nv) == 0  # nothing packed past the last position


@pytest.mark.parametrize("full", [True, False])
def test_paired_positions_are_the_documented_pairs(full):
    """The level at offset 16 pairs position i with i + NV/2; the kernel forms the mean, Sigma'
    diagonal and channel pairs from swapped inputs, so those pairs must stay paired."""
    nv, table = _tables()[full]
    slot = [(table >> (4 * pos)) & 15 for pos in range(nv)]
    pairs = {frozenset((slot[i], slot[i + nv // 2])) for i in range(nv // 2)}
    assert frozenset((0, 1)) in pairs  # (mean.x, mean.y)
    assert frozenset((2, 4)) in pairs  # (Sigma'.xx, Sigma'.yy)
    if full:
        for c, nrm in ((8, 12), (9, 13), (10, 14)):  # (colour, normal) channels
            assert frozenset((c, nrm)) in pairs
    else:
        assert frozenset((8, 9)) in pairs  # (red, green)
