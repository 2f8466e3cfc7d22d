// Warp-cooperative tile tests shared by the preprocess (tile counts and hit
// masks) and by the emission of instances for boxes of more than 32 tiles.
#pragma once

#include "ges_internal.cuh"

namespace ges {

// Tile tests of a warp's 32 entries, spread over the warp's lanes. Entry (lane) l
// owns the tests [excl_l, incl_l) of the warp's running count: the tiles of its
// box, row-major. Each round, lane j takes test j0 + j: the owner is found by a
// binary search over the inclusive prefix, the owner's ellipse and pixel box come
// by shuffle, and the round's hits are one ballot. A splat whose box spans
// thousands of tiles then costs its warp a share of rounds instead of one lane
// testing every tile while the other 31 wait. The test is tile_hit on the tile's
// pixel-centre rectangle clipped to the box, as in a per-entry loop over the box.
struct TileJob {
    float u, v, a, b, c, ia, ic, qm;
    uint32_t xs, ys;  // x0 | x1 << 16, y0 | y1 << 16 (pixel box, non-empty)
    uint32_t nbox;    // tiles in the box (0: nothing to test)
};

// Per-warp shared-memory table of the warp's jobs: 32 x 3 uint4 (48 B per lane).
constexpr int kJobWords = 3;

// on_round(hits, lo, len, first, tx, ty, owner, hit) is called by every lane once
// per round: hits = the round's ballot; this lane's own tests in the round are the
// ballot bits [lo, lo + len) and are tests first.. of its box (len 0: none);
// (tx, ty, owner, hit) describe the test this lane ran (hit false if none).
// jobs: the warp's table (kJobWords * 32 uint4 of shared memory): each lane publishes its
// ellipse, pixel box, first test index and a multiplier for dividing by its box width once,
// and each round reads its owner's from there.
template <class OnRound>
__device__ __forceinline__ void warp_tile_rounds(const TileJob &J, int lane, int lw, int lh, int tw, int th,
                                                 uint4 *jobs, OnRound &&on_round) {
    constexpr uint32_t FULL = 0xffffffffu;
    uint32_t incl = J.nbox;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t wtotal = __shfl_sync(FULL, incl, 31);
    const uint32_t excl = incl - J.nbox;
    if (wtotal == 0) return;  // warp-uniform
    {
        // k / rw for the box's test index k: q = umulhi(k, m) with m = floor((2^32 - 1) / rw) + 1
        // is floor(k / rw) or one more (m rw >= 2^32 and m <= (2^32 - 1) / rw + 1); width 1 aside
        const uint32_t rw = J.nbox ? (uint32_t)(((int)(J.xs >> 16) >> lw) - ((int)(J.xs & 0xffffu) >> lw) + 1) : 1u;
        const uint32_t m = rw > 1u ? 0xffffffffu / rw + 1u : 0u;
        __syncwarp();  // an earlier use of the table is over
        jobs[kJobWords * lane + 0] = make_uint4(__float_as_uint(J.u), __float_as_uint(J.v), __float_as_uint(J.a),
                                                __float_as_uint(J.b));
        jobs[kJobWords * lane + 1] = make_uint4(__float_as_uint(J.c), __float_as_uint(J.ia), __float_as_uint(J.ic),
                                                __float_as_uint(J.qm));
        jobs[kJobWords * lane + 2] = make_uint4(J.xs, J.ys, excl, m);
        __syncwarp();
    }
    for (uint32_t j0 = 0; j0 < wtotal; j0 += 32) {
        const uint32_t j = j0 + (uint32_t)lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t p = __shfl_sync(FULL, incl, owner + step - 1);
            if (p <= j) owner += step;
        }
        const uint4 w0 = jobs[kJobWords * owner + 0], w1 = jobs[kJobWords * owner + 1],
                    w2 = jobs[kJobWords * owner + 2];
        const float u = __uint_as_float(w0.x), v = __uint_as_float(w0.y);
        const float ca = __uint_as_float(w0.z), cb = __uint_as_float(w0.w);
        const float cc = __uint_as_float(w1.x), ia = __uint_as_float(w1.y);
        const float ic = __uint_as_float(w1.z), qm = __uint_as_float(w1.w);
        const uint32_t xs = w2.x, ys = w2.y, o_excl = w2.z, m = w2.w;
        bool hit = false;
        int tx = 0, ty = 0;
        if (j < wtotal) {
            const int x0 = (int)(xs & 0xffffu), x1 = (int)(xs >> 16);
            const int y0 = (int)(ys & 0xffffu), y1 = (int)(ys >> 16);
            const int tx0 = x0 >> lw, ty0 = y0 >> lh;
            const uint32_t rw = (uint32_t)((x1 >> lw) - tx0 + 1);
            const uint32_t k = j - o_excl;
            uint32_t row = rw > 1u ? __umulhi(k, m) : k;
            if ((uint64_t)row * rw > k) --row;
            tx = tx0 + (int)(k - row * rw);
            ty = ty0 + (int)row;
            const int px0 = max(tx * tw, x0), px1 = min(tx * tw + tw - 1, x1);
            const int py0 = max(ty * th, y0), py1 = min(ty * th + th - 1, y1);
            hit = tile_hit(u, v, ca, cb, cc, ia, ic, qm, px0, px1, py0, py1);
        }
        const uint32_t hits = __ballot_sync(FULL, hit);
        const uint32_t lo = max(excl, j0), hi = min(incl, j0 + 32u);
        const bool mine = lo < hi;
        // one call by every lane (on_round may shuffle)
        on_round(hits, mine ? lo - j0 : 0u, mine ? hi - lo : 0u, mine ? lo - excl : 0u, tx, ty, (uint32_t)owner, hit);
    }
}

}  // namespace ges
