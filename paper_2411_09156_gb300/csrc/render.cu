// S6 forward compositing and S7 backward replay.
//
// One CTA per tile (persistent CTAs take tiles from a longest-first queue). Each
// warp owns a compact 8x4 block of the tile's pixels and walks the tile's
// depth-sorted list on its own, 32 entries at a time: every lane loads one
// record, tests whether that splat's support can reach any pixel of the warp's
// block (the exact ellipse-rectangle test of the binning, with a margin), and the
// warp then evaluates only the splats that can (ballot + find-first-set), reading
// them from a per-warp shared-memory slot. Warps never wait for each other: a
// warp stops as soon as its own pixels reach the transmittance cutoff (forward)
// or its last contributor (backward), and the records shared by the warps of a
// tile are served from L1/L2. Each warp prefetches the records `batch` entries
// ahead of the chunk it evaluates into L2.
//
// The backward replays the list front to back from the stored t_final and
// `last` (no per-pixel lists), and reduces each splat's gradient values (14, or
// 10 without depth and normal) across the warp with a transposing butterfly
// (15 or 12 shuffles in all, instead of 5 per value) before one lane of each
// pair issues its value's FP32 atomic into the splat's 64-byte accumulator.
#include "ges_internal.cuh"

namespace ges {

// Next work item of a warp: a tile and the 8x4 sub-block of it that the warp
// renders. Plain launch: CTA = tile, warp w takes sub-block w. Persistent launch:
// each warp takes the next (tile, sub-block) item of the longest-first queue with
// its own atomic, so no warp waits for another.
__device__ __forceinline__ bool next_item(const uint32_t *queue, uint32_t *counter, uint32_t n_tiles, int nw, int it,
                                          int warp, int lane, uint32_t &tile, int &sb) {
    if (queue) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_tiles * (uint32_t)nw) return false;
        tile = queue[item / (uint32_t)nw];
        sb = (int)(item % (uint32_t)nw);
        return true;
    }
    if (it > 0) return false;
    tile = blockIdx.x;
    sb = warp;
    return true;
}

__device__ __forceinline__ int view_of_tile(const ViewSet &V, uint32_t tile) {
    int v = 0;
    while (v + 1 < V.n_views && (int)tile >= V.tile_base[v + 1]) ++v;
    return v;
}

constexpr uint32_t kNone = 0xffffffffu;

__device__ __forceinline__ uint32_t entry_or_none(const uint32_t *inst_entry, uint32_t idx, uint32_t end) {
    return idx < end ? __ldg(inst_entry + idx) : kNone;
}

// Warp footprint inside a tile: 8 x 4 pixels.
constexpr int kWarpW = 8, kWarpH = 4;
// A staged record takes 4 float4 and is padded to 5: a quarter-warp's 16-byte stores then fall in
// 8 distinct groups of 4 banks (lane * 5 mod 8) instead of 2 (lane * 4 mod 8).
constexpr int kSlotVec = 5;

template <int TW>
__device__ __forceinline__ void warp_pixel(int sb, int lane, int &lx, int &ly, int &wx0, int &wy0) {
    constexpr int WPR = TW / kWarpW;
    wx0 = (sb % WPR) * kWarpW;
    wy0 = (sb / WPR) * kWarpH;
    lx = wx0 + (lane & 7);
    ly = wy0 + (lane >> 3);
}

// Can the support Q <= q_cut of a splat with centre (u, v) and conic (a, b, c)
// reach the rectangle of pixel centres [rx0, rx1] x [ry0, ry1]? The minimum of
// the convex Q over the rectangle is 0 if it holds the centre, else it lies on
// an edge at the clamped 1-D minimiser. qm carries a margin (1 + 2^-10) that
// absorbs the rounding of this estimate, so the test never drops a pixel that
// the per-pixel evaluation would blend.
__device__ __forceinline__ bool warp_may_hit(float u, float v, float a, float b, float c, float qm, float rx0,
                                             float rx1, float ry0, float ry1) {
    const float X0 = rx0 - u, X1 = rx1 - u, Y0 = ry0 - v, Y1 = ry1 - v;
    if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return true;
    const float ia = __frcp_rn(a), ic = __frcp_rn(c), b2 = b + b;
    auto q = [&](float X, float Y) { return fmaf(a * X, X, fmaf(b2 * X, Y, c * Y * Y)); };
    float best = q(X0, fminf(fmaxf(-b * X0 * ic, Y0), Y1));
    best = fminf(best, q(X1, fminf(fmaxf(-b * X1 * ic, Y0), Y1)));
    best = fminf(best, q(fminf(fmaxf(-b * Y0 * ia, X0), X1), Y0));
    best = fminf(best, q(fminf(fmaxf(-b * Y1 * ia, X0), X1), Y1));
    return best <= qm;
}

// Debug build: an entry read from a tile list must name one of the n_entries (view, splat)
// records; if it does not, the error word records GES_ERR_BOUNDS and the entry is skipped.
__device__ __forceinline__ bool entry_ok(uint32_t e, uint32_t n_entries, uint32_t *err) {
#ifdef GES_DEBUG
    if (e >= n_entries) {
        set_error(err, kErrBounds);
        return false;
    }
#endif
    return true;
}

// The cull vectors (u, v, a, b), (c, q_cut, beta/2, o) of record e, or zeros for no entry.
__device__ __forceinline__ void load_cull_vectors(const float4 *rec, uint32_t e, uint32_t n_entries, uint32_t *err,
                                                  float4 &r0, float4 &r1) {
    r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    r1 = r0;
    if (e == kNone || !entry_ok(e, n_entries, err)) return;
    const float4 *r = rec + 4 * (size_t)e;
    r0 = __ldg(r);
    r1 = __ldg(r + 1);
}

// Tests record e (its cull vectors r0, r1 already loaded) against the warp's block and, if it can
// contribute, stores it (with 2b in place of b) into the warp's slot `lane`.
__device__ __forceinline__ bool cull_stage(const float4 *rec, uint32_t e, uint32_t n_entries, uint32_t *err, float4 r0,
                                           const float4 r1, float rx0, float rx1, float ry0, float ry1,
                                           float4 (*slot)[kSlotVec], int lane) {
    if (e == kNone || !entry_ok(e, n_entries, err)) return false;
    if (!warp_may_hit(r0.x, r0.y, r0.z, r0.w, r1.x, r1.y * kSupportMargin, rx0, rx1, ry0, ry1)) return false;
    const float4 *r = rec + 4 * (size_t)e;
    r0.w = r0.w + r0.w;
    slot[lane][0] = r0;
    slot[lane][1] = r1;
    slot[lane][2] = __ldg(r + 2);
    slot[lane][3] = __ldg(r + 3);
    return true;
}

// Loads record e, tests it against the warp's block and, if it can contribute,
// stores it (with 2b in place of b) into the warp's slot `lane`.
__device__ __forceinline__ bool load_cull_stage(const float4 *rec, uint32_t e, uint32_t n_entries, uint32_t *err,
                                                float rx0, float rx1, float ry0, float ry1, float4 (*slot)[kSlotVec],
                                                int lane) {
    if (e == kNone || !entry_ok(e, n_entries, err)) return false;
    const float4 *r = rec + 4 * (size_t)e;
    float4 r0 = __ldg(r);
    const float4 r1 = __ldg(r + 1);
    if (!warp_may_hit(r0.x, r0.y, r0.z, r0.w, r1.x, r1.y * kSupportMargin, rx0, rx1, ry0, ry1)) return false;
    r0.w = r0.w + r0.w;
    slot[lane][0] = r0;
    slot[lane][1] = r1;
    slot[lane][2] = __ldg(r + 2);
    slot[lane][3] = __ldg(r + 3);
    return true;
}

// DN: the depth and normal outputs are wanted; without them (the training step renders for a
// loss on the colour) their accumulations drop out.
template <int TW, int TH, bool DN>
__global__ void __launch_bounds__(TW *TH) k_render_fwd(const FwdArgs a) {
    constexpr int NW = TW * TH / 32;
    __shared__ float4 s_rec[NW][32][kSlotVec];  // per-warp slot of the current chunk's records
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4(*slot)[kSlotVec] = s_rec[warp];
    const uint32_t ahead = (uint32_t)a.batch;
    uint32_t tile;
    int sb;
    for (int it = 0; next_item(a.queue, a.counter, (uint32_t)a.V.n_tiles, NW, it, warp, lane, tile, sb); ++it) {
        int lx, ly, wx0, wy0;
        warp_pixel<TW>(sb, lane, lx, ly, wx0, wy0);
        const int v = view_of_tile(a.V, tile);
        const int lt = (int)tile - a.V.tile_base[v];
        const int tiles_x = a.V.tiles_x[v];
        const int W = a.V.width[v], H = a.V.height[v];
        const int tx0 = (lt % tiles_x) * TW, ty0 = (lt / tiles_x) * TH;
        const int px = tx0 + lx, py = ty0 + ly;
        const bool inside = px < W && py < H;
        const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
        const float rx0 = (float)(tx0 + wx0) + 0.5f, rx1 = rx0 + (float)(kWarpW - 1);
        const float ry0 = (float)(ty0 + wy0) + 0.5f, ry1 = ry0 + (float)(kWarpH - 1);
        const uint2 rg = a.ranges[tile];
        float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, N0 = 0.f, N1 = 0.f, N2 = 0.f;
        uint32_t cnt = 0, last = rg.x, stop = rg.y, events = 0;
        bool done = !inside;
        // software pipeline over 32-entry chunks: entry indices are read two chunks ahead and the
        // cull vectors (r0, r1) of the next chunk are in flight while this chunk is evaluated
        uint32_t e_cur = entry_or_none(a.inst_entry, rg.x + lane, rg.y);
        uint32_t e_nxt = entry_or_none(a.inst_entry, rg.x + 32 + lane, rg.y);
        uint32_t e_pf = entry_or_none(a.inst_entry, rg.x + ahead + lane, rg.y);
        float4 q0, q1;
        load_cull_vectors(a.rec, e_cur, a.n_entries, a.err, q0, q1);
        for (uint32_t c0 = rg.x; c0 < rg.y; c0 += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            if (e_pf != kNone && entry_ok(e_pf, a.n_entries, a.err)) prefetch_l2(a.rec + 4 * (size_t)e_pf);
            e_pf = entry_or_none(a.inst_entry, c0 + 32 + ahead + lane, rg.y);
            const uint32_t e_nn = entry_or_none(a.inst_entry, c0 + 64 + lane, rg.y);
            float4 n0, n1;
            load_cull_vectors(a.rec, e_nxt, a.n_entries, a.err, n0, n1);
            const bool hit = cull_stage(a.rec, e_cur, a.n_entries, a.err, q0, q1, rx0, rx1, ry0, ry1, slot, lane);
            e_cur = e_nxt;
            e_nxt = e_nn;
            q0 = n0;
            q1 = n1;
            uint32_t mask = __ballot_sync(0xffffffffu, hit);
            events += __popc(mask);
            __syncwarp();
            while (mask) {
                const int bit = __ffs(mask) - 1;
                mask &= mask - 1;
                if (done) continue;
                const float4 r0 = slot[bit][0], r1 = slot[bit][1];
                PairEval pe;
                if (!eval_pair(fpx - r0.x, fpy - r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, a.alpha_max, a.alpha_min,
                               pe))
                    continue;
                const float Tn = __fmul_rn(T, __fsub_rn(1.f, pe.alpha));
                if (Tn < a.t_min) { done = true; stop = c0 + (uint32_t)bit + 1; continue; }
                const float w = __fmul_rn(pe.alpha, T);
                const float4 r2 = slot[bit][2], r3 = slot[bit][3];
                C0 = __fmaf_rn(w, r2.x, C0);
                C1 = __fmaf_rn(w, r2.y, C1);
                C2 = __fmaf_rn(w, r2.z, C2);
                if (DN) {
                    D = __fmaf_rn(w, r2.w, D);
                    N0 = __fmaf_rn(w, r3.x, N0);
                    N1 = __fmaf_rn(w, r3.y, N1);
                    N2 = __fmaf_rn(w, r3.z, N2);
                }
                T = Tn;
                ++cnt;
                last = c0 + (uint32_t)bit + 1;
            }
            __syncwarp();
        }
        if (inside) {
            const long long P = (long long)W * H;
            const long long pix = (long long)py * W + px;
            const long long g = a.V.pix_base[v] + pix;
            float *col = a.color + 3 * a.V.pix_base[v] + pix;
            col[0] = __fmaf_rn(T, a.bg[0], C0);
            col[P] = __fmaf_rn(T, a.bg[1], C1);
            col[2 * P] = __fmaf_rn(T, a.bg[2], C2);
            if (DN && a.depth) a.depth[g] = D;
            a.alpha[g] = 1.f - T;
            if (DN && a.normal) {
                float *nrm = a.normal + 3 * a.V.pix_base[v] + pix;
                nrm[0] = N0; nrm[P] = N1; nrm[2 * P] = N2;
            }
            a.t_final[g] = T;
            a.last[g] = last;
            a.n_contrib[g] = cnt;
            if (a.n_eval) a.n_eval[g] = stop - rg.x;
        }
        if (a.n_events && lane == 0) atomicAdd(a.n_events, (unsigned long long)events);
    }
}

// Warp sum of NV values by recursive halving. At the level with lane offset D a lane whose bit D
// is clear keeps the first H = ceil(n / 2) of its n values and the other lane the rest (padded
// with a zero when n is odd), each adding what its partner sends: NV - 1 + ... shuffles in all
// (16 for 16 values, 12 for 10). After the levels 16, 8, 4, 2 each lane pair holds one value
// index, reduce_label(NV, lane), or -1; the last level sums the pair.
template <int D, int N>
__device__ __forceinline__ void halve(float *g, int lane) {
    constexpr int H = (N + 1) / 2;
    const bool up = lane & D;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float rest = (H + i < N) ? g[H + i] : 0.f;
        const float send = up ? g[i] : rest;
        const float keep = up ? rest : g[i];
        g[i] = keep + __shfl_xor_sync(0xffffffffu, send, D);
    }
}

template <int NV>
__device__ __forceinline__ float warp_reduce_n(float (&g)[NV], int lane) {
    static_assert(NV >= 9 && NV <= 16, "four halvings leave one value");
    constexpr int N1 = (NV + 1) / 2, N2 = (N1 + 1) / 2, N3 = (N2 + 1) / 2;
    halve<16, NV>(g, lane);
    halve<8, N1>(g, lane);
    halve<4, N2>(g, lane);
    halve<2, N3>(g, lane);
    return g[0] + __shfl_xor_sync(0xffffffffu, g[0], 1);
}

// warp_reduce_n<NV> with the level at offset 16 given as the values each lane keeps and sends
// (NV even): keep[i] and send[i] are positions i and i + NV/2 in the order of the lane's half.
template <int NV>
__device__ __forceinline__ float warp_reduce_split(const float (&keep)[NV / 2], const float (&send)[NV / 2],
                                                   int lane) {
    static_assert(NV % 2 == 0 && NV >= 10 && NV <= 16, "three halvings after the split leave one value");
    constexpr int N1 = NV / 2, N2 = (N1 + 1) / 2, N3 = (N2 + 1) / 2;
    float g[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) g[i] = keep[i] + __shfl_xor_sync(0xffffffffu, send[i], 16);
    halve<8, N1>(g, lane);
    halve<4, N2>(g, lane);
    halve<2, N3>(g, lane);
    return g[0] + __shfl_xor_sync(0xffffffffu, g[0], 1);
}

// The value index that lane's pair holds after warp_reduce_n<NV>, or -1 (a padding zero).
__device__ __forceinline__ int reduce_label(int nv, int lane) {
    int start = 0, valid = nv, n = nv;
    for (int d = 16; d >= 2; d >>= 1) {
        const int h = (n + 1) / 2;
        if (lane & d) { start += h; valid = valid > h ? valid - h : 0; }
        else valid = valid < h ? valid : h;
        n = h;
    }
    return valid > 0 ? start : -1;
}

// FULL: the depth and normal outputs have upstream gradients too; without them (a loss on the
// colour, the training step) their channels drop out of the replay.
template <int TW, int TH, bool FULL>
__global__ void __launch_bounds__(TW *TH) k_render_bwd(const BwdArgs a) {
    constexpr int NW = TW * TH / 32;
    __shared__ float4 s_rec[NW][32][kSlotVec];
    __shared__ uint32_t s_ent[NW][32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float4(*slot)[kSlotVec] = s_rec[warp];
    uint32_t *went = s_ent[warp];
    const uint32_t ahead = (uint32_t)a.batch;
    const float ln2 = 0.69314718055994531f;
    // The gradient values a pair contributes, in reduction order: the level at lane offset 16 pairs
    // position i with i + NV/2, and the pairs are chosen so that few of them need a per-event swap
    // (see the event body):
    //   FULL:   mean.x  S.xx  S.xy     red    green  blue   beta  |  mean.y  S.yy  opacity  n.x  n.y  n.z  depth
    //   colour: mean.x  S.xx  S.xy     red    blue                |  mean.y  S.yy  opacity  green  beta
    // (S = Sigma'). Position p goes to slot (kSlots >> 4p) & 15 of the splat's 16-float
    // accumulator: 0-1 mean, 2-4 Sigma' xx xy yy, 5 opacity, 6 beta, 7 depth, 8-10 colour,
    // 12-14 normal (slots 11 and 15, and without FULL 7 and 12-14, stay 0). After the reduction
    // this lane's pair holds position `lab`.
    constexpr int NV = FULL ? 14 : 10;
    constexpr int H1 = NV / 2;
    constexpr unsigned long long kSlots = FULL ? 0x7EDC5416A98320ull : 0x69541A8320ull;
    const int lab = reduce_label(NV, lane);
    const int gslot = lab < 0 ? -1 : (int)((kSlots >> (4 * lab)) & 15u);
    const bool writer = (lane & 1) == 0 && gslot >= 0;
    const bool up16 = (lane & 16) != 0;
    uint32_t tile;
    int sb;
    for (int it = 0; next_item(a.queue, a.counter, (uint32_t)a.V.n_tiles, NW, it, warp, lane, tile, sb); ++it) {
        int lx, ly, wx0, wy0;
        warp_pixel<TW>(sb, lane, lx, ly, wx0, wy0);
        const int v = view_of_tile(a.V, tile);
        const int lt = (int)tile - a.V.tile_base[v];
        const int tiles_x = a.V.tiles_x[v];
        const int W = a.V.width[v], H = a.V.height[v];
        const int tx0 = (lt % tiles_x) * TW, ty0 = (lt / tiles_x) * TH;
        const int px = tx0 + lx, py = ty0 + ly;
        const bool inside = px < W && py < H;
        const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
        const float rx0 = (float)(tx0 + wx0) + 0.5f, rx1 = rx0 + (float)(kWarpW - 1);
        const float ry0 = (float)(ty0 + wy0) + 0.5f, ry1 = ry0 + (float)(kWarpH - 1);
        const uint2 rg = a.ranges[tile];
        // per-pixel forward results F_k and upstream gradients g_k of the 7 blended
        // channels (colour, depth, normal), and g_alpha T_final
        float Cf0 = 0.f, Cf1 = 0.f, Cf2 = 0.f, Df = 0.f, Nf0 = 0.f, Nf1 = 0.f, Nf2 = 0.f, gAT = 0.f;
        float gC0 = 0.f, gC1 = 0.f, gC2 = 0.f, gD = 0.f, gN0 = 0.f, gN1 = 0.f, gN2 = 0.f;
        uint32_t lp = rg.x;
        if (inside) {
            const long long P = (long long)W * H;
            const long long pix = (long long)py * W + px;
            const long long g = a.V.pix_base[v] + pix;
            const long long c3 = 3 * a.V.pix_base[v] + pix;
            lp = a.last[g];
#ifdef GES_DEBUG
            if (lp < rg.x || lp > rg.y) {  // the replay stays inside this tile's list
                set_error(a.err, kErrBounds);
                lp = rg.x;
            }
#endif
            if (a.g_color) {
                gC0 = a.g_color[c3]; gC1 = a.g_color[c3 + P]; gC2 = a.g_color[c3 + 2 * P];
                Cf0 = a.color[c3]; Cf1 = a.color[c3 + P]; Cf2 = a.color[c3 + 2 * P];
            }
            if (FULL && a.g_depth) { gD = a.g_depth[g]; Df = a.depth[g]; }
            if (a.g_alpha) gAT = a.g_alpha[g] * a.t_final[g];
            if (FULL && a.g_normal) {
                gN0 = a.g_normal[c3]; gN1 = a.g_normal[c3 + P]; gN2 = a.g_normal[c3 + 2 * P];
                Nf0 = a.normal[c3]; Nf1 = a.normal[c3 + P]; Nf2 = a.normal[c3 + 2 * P];
            }
        }
        // the per-pixel factors of the channel pairs (red, n.x), (green, n.y), (blue, n.z) (FULL) or
        // (red, green) in kept / sent order for the level at offset 16: a lane with bit 16 clear keeps
        // the first of a pair and sends the second, the others the reverse
        const float kc0 = FULL ? (up16 ? gN0 : gC0) : (up16 ? gC1 : gC0);
        const float sc0 = FULL ? (up16 ? gC0 : gN0) : (up16 ? gC0 : gC1);
        const float kc1 = up16 ? gN1 : gC1, sc1 = up16 ? gC1 : gN1;
        const float kc2 = up16 ? gN2 : gC2, sc2 = up16 ? gC2 : gN2;
        const uint32_t wend = __reduce_max_sync(0xffffffffu, lp);  // this warp replays [rg.x, wend)
        // transmittance before splat i and the channels accumulated up to and including
        // splat i, A_k, in the forward pass's operation order: F_k - A_k, the part of the
        // pixel behind splat i, is then exact at the last splat and carries only the
        // rounding of the later steps
        float T = 1.f, Ca0 = 0.f, Ca1 = 0.f, Ca2 = 0.f, Da = 0.f, Na0 = 0.f, Na1 = 0.f, Na2 = 0.f;
        uint32_t e_cur = entry_or_none(a.inst_entry, rg.x + lane, wend);
        uint32_t e_pf = entry_or_none(a.inst_entry, rg.x + ahead + lane, wend);
        for (uint32_t c0 = rg.x; c0 < wend; c0 += 32) {
            if (e_pf != kNone && entry_ok(e_pf, a.n_entries, a.err)) prefetch_l2(a.rec + 4 * (size_t)e_pf);
            e_pf = entry_or_none(a.inst_entry, c0 + 32 + ahead + lane, wend);
            const uint32_t e_nxt = entry_or_none(a.inst_entry, c0 + 32 + lane, wend);
            const bool hit = load_cull_stage(a.rec, e_cur, a.n_entries, a.err, rx0, rx1, ry0, ry1, slot, lane);
            if (hit) went[lane] = e_cur;
            e_cur = e_nxt;
            uint32_t mask = __ballot_sync(0xffffffffu, hit);
            __syncwarp();
            while (mask) {
                const int bit = __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 r0 = slot[bit][0], r1 = slot[bit][1];
                const float dx = fpx - r0.x, dy = fpy - r0.y;
                PairEval pe;
                const bool contrib =
                    eval_pair_all(dx, dy, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, a.alpha_max, a.alpha_min, pe) &&
                    c0 + (uint32_t)bit < lp;
                // Warp-uniform skip when no lane blends this splat; otherwise the body runs branch-free on
                // every lane: a lane that does not blend takes alpha = 0, which leaves T and the running
                // sums exactly as they were, and its values are selected to zero.
                if (!__any_sync(0xffffffffu, contrib)) continue;
                float keep[H1], send[H1];
                {
                    const float4 r2 = slot[bit][2], r3 = slot[bit][3];
                    const float al = contrib ? pe.alpha : 0.f;  // 0: every running sum below is unchanged
                    const float w = __fmul_rn(al, T);
                    Ca0 = __fmaf_rn(w, r2.x, Ca0);
                    Ca1 = __fmaf_rn(w, r2.y, Ca1);
                    Ca2 = __fmaf_rn(w, r2.z, Ca2);
                    // d out / d alpha_i = T_i sum_k g_k c_ik - (sum_k g_k (F_k - A_k) - g_alpha T_final) / (1 - alpha_i)
                    float gc = gC0 * r2.x + gC1 * r2.y + gC2 * r2.z;
                    float behind = gC0 * (Cf0 - Ca0) + gC1 * (Cf1 - Ca1) + gC2 * (Cf2 - Ca2);
                    if (FULL) {
                        Da = __fmaf_rn(w, r2.w, Da);
                        Na0 = __fmaf_rn(w, r3.x, Na0);
                        Na1 = __fmaf_rn(w, r3.y, Na1);
                        Na2 = __fmaf_rn(w, r3.z, Na2);
                        gc = gc + gD * r2.w + gN0 * r3.x + gN1 * r3.y + gN2 * r3.z;
                        behind = behind + gD * (Df - Da) + gN0 * (Nf0 - Na0) + gN1 * (Nf1 - Na1) +
                                 gN2 * (Nf2 - Na2);
                    }
                    const float dal = contrib ? T * gc - (behind - gAT) * rcp_approx(1.f - al) : 0.f;
                    T = __fmul_rn(T, __fsub_rn(1.f, al));
                    const float o = r1.w, hb = r1.z;
                    const bool unclamped = contrib && pe.alpha_raw < a.alpha_max;
                    const float gop = unclamped ? dal * pe.G : 0.f;
                    const float gG = unclamped ? dal * o : 0.f;
                    // G = exp(-p/2), p = Q^(beta/2): dG/dQ = -(beta/4) (p/Q) G, dG/dbeta = -(1/4) p ln(Q) G
                    const bool qpos = contrib && pe.Q > 0.f;
                    const float gp = gG * pe.p * pe.G;
                    const float nq = qpos ? 0.5f * hb * gp * rcp_approx(pe.Q) : 0.f;  // -dL/dQ
                    const float gbeta = qpos ? -0.25f * ln2 * gp * pe.lq : 0.f;
                    // Q = d^T C d with C = Sigma'^-1 and d = pixel - mean; with m = C d:
                    // dQ/dmean = -2 m and dQ/dSigma' = -m m^T (accumulated directly:
                    // going through the conic gradient would cancel for thin splats)
                    const float mx = fmaf(r0.z, dx, 0.5f * r0.w * dy), my = fmaf(0.5f * r0.w, dx, r1.x * dy);
                    // pairs (2 qx, 2 qy) and (qx mx, qy my), q = -dL/dQ m, from m in kept / sent order;
                    // qx my = qy mx is S.xy either way. The channel pairs take their per-pixel factors
                    // in that order already; the rest are swapped here.
                    const float mk = up16 ? my : mx, ms = up16 ? mx : my;
                    const float qk = nq * mk, qs = nq * ms;
                    keep[0] = 2.f * qk; send[0] = 2.f * qs;
                    keep[1] = qk * mk; send[1] = qs * ms;
                    const float sxy = qk * ms;
                    keep[2] = up16 ? gop : sxy; send[2] = up16 ? sxy : gop;
                    keep[3] = kc0 * w; send[3] = sc0 * w;
                    if (FULL) {
                        keep[FULL ? 4 : 0] = kc1 * w; send[FULL ? 4 : 0] = sc1 * w;
                        keep[FULL ? 5 : 0] = kc2 * w; send[FULL ? 5 : 0] = sc2 * w;
                        const float gdep = gD * w;
                        keep[FULL ? 6 : 0] = up16 ? gdep : gbeta; send[FULL ? 6 : 0] = up16 ? gbeta : gdep;
                    } else {
                        const float cb = gC2 * w;
                        keep[4] = up16 ? gbeta : cb; send[4] = up16 ? cb : gbeta;
                    }
                }
                const float sum = warp_reduce_split<NV>(keep, send, lane);
                if (writer) atomicAdd(a.g2d + 16 * (size_t)went[bit] + gslot, sum);
            }
            __syncwarp();
        }
    }
}

// Persistent grid: as many CTAs of `kernel` as fit on every SM at once.
template <class K>
static int persistent_grid(K kernel, int threads) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, 0);
    if (per < 1) per = 1;
    return sms * per;
}

template <int TW, int TH, bool DN>
static cudaError_t launch_fwd_t(const FwdArgs &a, cudaStream_t s) {
    int grid = a.V.n_tiles;
    if (a.queue) grid = min(grid, persistent_grid(k_render_fwd<TW, TH, DN>, TW * TH));
    if (grid <= 0) return cudaSuccess;
    k_render_fwd<TW, TH, DN><<<grid, TW * TH, 0, s>>>(a);
    return cudaGetLastError();
}


template <int TW, int TH, bool FULL>
static cudaError_t launch_bwd_t(const BwdArgs &a, cudaStream_t s) {
    int grid = a.V.n_tiles;
    if (a.queue) grid = min(grid, persistent_grid(k_render_bwd<TW, TH, FULL>, TW * TH));
    if (grid <= 0) return cudaSuccess;
    k_render_bwd<TW, TH, FULL><<<grid, TW * TH, 0, s>>>(a);
    return cudaGetLastError();
}

bool tile_shape_supported(int tw, int th) {
    return (tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 32 && th == 8) || (tw == 8 && th == 32) ||
           (tw == 16 && th == 8) || (tw == 8 && th == 16);
}

cudaError_t launch_render_fwd(const FwdArgs &a, cudaStream_t s) {
    const int tw = a.V.tile_w, th = a.V.tile_h;
    const bool dn = a.depth != nullptr || a.normal != nullptr;
    if (tw == 16 && th == 16) return dn ? launch_fwd_t<16, 16, true>(a, s) : launch_fwd_t<16, 16, false>(a, s);
    if (tw == 8 && th == 8) return dn ? launch_fwd_t<8, 8, true>(a, s) : launch_fwd_t<8, 8, false>(a, s);
    if (tw == 8 && th == 32) return dn ? launch_fwd_t<8, 32, true>(a, s) : launch_fwd_t<8, 32, false>(a, s);
    if (tw == 16 && th == 8) return dn ? launch_fwd_t<16, 8, true>(a, s) : launch_fwd_t<16, 8, false>(a, s);
    if (tw == 8 && th == 16) return dn ? launch_fwd_t<8, 16, true>(a, s) : launch_fwd_t<8, 16, false>(a, s);
    return dn ? launch_fwd_t<32, 8, true>(a, s) : launch_fwd_t<32, 8, false>(a, s);
}

cudaError_t launch_render_bwd(const BwdArgs &a, cudaStream_t s) {
    const int tw = a.V.tile_w, th = a.V.tile_h;
    const bool full = a.g_depth != nullptr || a.g_normal != nullptr;
    if (tw == 16 && th == 16) return full ? launch_bwd_t<16, 16, true>(a, s) : launch_bwd_t<16, 16, false>(a, s);
    if (tw == 8 && th == 8) return full ? launch_bwd_t<8, 8, true>(a, s) : launch_bwd_t<8, 8, false>(a, s);
    if (tw == 8 && th == 32) return full ? launch_bwd_t<8, 32, true>(a, s) : launch_bwd_t<8, 32, false>(a, s);
    if (tw == 16 && th == 8) return full ? launch_bwd_t<16, 8, true>(a, s) : launch_bwd_t<16, 8, false>(a, s);
    if (tw == 8 && th == 16) return full ? launch_bwd_t<8, 16, true>(a, s) : launch_bwd_t<8, 16, false>(a, s);
    return full ? launch_bwd_t<32, 8, true>(a, s) : launch_bwd_t<32, 8, false>(a, s);
}

}  // namespace ges
