// Internal definitions shared by the CUDA translation units of libges.so.
// Nothing here is part of the C ABI (include/ges.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "ges.h"

namespace ges {

// NVTX range named after the C-ABI entry point, for timelines of profiling tools (a no-op
// when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define GES_RANGE() ::ges::NvtxRange ges_range_(__func__)

constexpr int kMaxViews = GES_MAX_VIEWS;
constexpr uint32_t kCulledKey = 0xffffffffu;
// Widening of the support used for binning only: q_cut * (1 + 2^-10).
constexpr float kSupportMargin = 1.0009765625f;
// -1/2 log2(e): exp(-x/2) = exp2(kNegHalfLog2e * x).
constexpr float kNegHalfLog2e = -0.72134752044448170f;

// Error-word bits (1 << ges_status).
constexpr uint32_t kErrCapacity = 1u << GES_ERR_CAPACITY;
constexpr uint32_t kErrNumeric = 1u << GES_ERR_NUMERIC;
constexpr uint32_t kErrBounds = 1u << GES_ERR_BOUNDS;

// Per-view constants handed to every kernel by value.
struct ViewSet {
    int n_views;
    int n_tiles;                       // total over views
    int tile_w, tile_h;
    int width[kMaxViews], height[kMaxViews];
    int tiles_x[kMaxViews];
    int tile_base[kMaxViews + 1];      // prefix of tile counts
    long long pix_base[kMaxViews + 1]; // prefix of pixel counts
    float fx[kMaxViews], fy[kMaxViews], cx[kMaxViews], cy[kMaxViews];
    float vm[kMaxViews][12];
    float znear[kMaxViews];
    float limx[kMaxViews], limy[kMaxViews];  // Jacobian clamp on X/Z and Y/Z
    float campos[kMaxViews][3];              // camera centre = -R^T t
};

struct Params {
    int sh_degree;  // -1 or 0..3
    int n_coeffs;   // (deg+1)^2, or 1 for RGB
    int phi_mode;
    float rho, lowpass, alpha_min, alpha_max, t_min;
    float bg[3];
    int color_storage;  // colour input: 0 float32, 1 binary16, 2 bfloat16
};

// 16-bit colour value of storage type st (1 binary16, 2 bfloat16) widened to float32 (exact).
__device__ __forceinline__ float widen16(uint32_t h, int st) {
    return st == 1 ? __half2float(__ushort_as_half((unsigned short)h)) : __uint_as_float(h << 16);
}

// Element q of a colour array of storage type st (0 float32, 1 binary16, 2 bfloat16), as float32.
__device__ __forceinline__ float ld_color(const void *base, int st, size_t q) {
    if (st == 0) return __ldg(static_cast<const float *>(base) + q);
    return widen16(__ldg(static_cast<const unsigned short *>(base) + q), st);
}

// Eight 16-bit colour values at a 16-byte aligned address, widened to float32.
__device__ __forceinline__ void ld_color8(const void *p, int st, float *out) {
    const uint4 u = __ldg(static_cast<const uint4 *>(p));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        out[2 * j] = widen16(w[j] & 0xffffu, st);
        out[2 * j + 1] = widen16(w[j] >> 16, st);
    }
}

// ------------------------------------------------------------------ layouts
// proj: [header 256 B][records nV x 64 B][binrec nV x 32 B][g2d nV x 64 B]
// header: u64 instance total at 0, u32 error word at 8.
struct ProjLayout {
    uint64_t records, binrec, g2d, bytes;
};

__host__ __device__ inline uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

inline ProjLayout proj_layout(int32_t n, int32_t n_views) {
    const uint64_t nv = (uint64_t)n * (uint64_t)n_views;
    ProjLayout L;
    L.records = 256;
    L.binrec = align256(L.records + nv * 64);
    L.g2d = align256(L.binrec + nv * 32);
    L.bytes = align256(L.g2d + nv * 64);
    return L;
}

// Radix sort / scan geometry.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per CTA
constexpr int kScanTile = 4096;
constexpr int kScanMaxPartials = 1024 * 16;

inline uint32_t ceil_div_u64(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

// bins: [header 256][dkey 2 x nV][dval 2 x nV][rank counts nV][rank info nV x 16][ikey 2 x cap]
//       [ival 2 x cap][ranges T x 8][queue T][hist 256 x nblk][partials]
// header: u32 n_inst (instances actually listed) at 0, u32 queue counters at 4 and 8, u64 count of
// the forward's warp-cull passes at 16 (written only when the forward is asked for n_eval).
struct BinsLayout {
    uint64_t dkey[2], dval[2], rcount, rinfo, ikey[2], ival[2], ranges, queue, hist, partials, bytes;
    uint32_t n_tiles;
    uint32_t nblk_entries, nblk_inst;  // radix CTAs for the depth sort and the tile sort
    int tile_passes;                   // 8-bit passes of the tile sort
};

inline int bits_for(uint32_t v) {  // bits needed to hold values 0..v-1
    int b = 0;
    while (b < 32 && (1ull << b) < (uint64_t)v) ++b;
    return b;
}

inline BinsLayout bins_layout(int32_t n, int32_t n_views, uint32_t n_tiles, uint64_t cap) {
    const uint64_t nv = (uint64_t)n * (uint64_t)n_views;
    BinsLayout L;
    L.n_tiles = n_tiles;
    uint64_t off = 256;
    for (int i = 0; i < 2; ++i) { L.dkey[i] = off; off = align256(off + nv * 4); }
    for (int i = 0; i < 2; ++i) { L.dval[i] = off; off = align256(off + nv * 4); }
    L.rcount = off; off = align256(off + nv * 4 + 4);
    L.rinfo = off; off = align256(off + nv * 16);
    for (int i = 0; i < 2; ++i) { L.ikey[i] = off; off = align256(off + cap * 4); }
    for (int i = 0; i < 2; ++i) { L.ival[i] = off; off = align256(off + cap * 4); }
    L.ranges = off; off = align256(off + (uint64_t)n_tiles * 8);
    L.queue = off; off = align256(off + (uint64_t)n_tiles * 4);
    L.nblk_entries = ceil_div_u64(nv > 0 ? nv : 1, kSortTile);
    L.nblk_inst = ceil_div_u64(cap > 0 ? cap : 1, kSortTile);
    uint32_t nblk = L.nblk_entries > L.nblk_inst ? L.nblk_entries : L.nblk_inst;
    L.hist = off; off = align256(off + (uint64_t)256 * nblk * 4);
    uint64_t scan_n = (uint64_t)256 * nblk;
    if (nv > scan_n) scan_n = nv;
    L.partials = off; off = align256(off + ((uint64_t)ceil_div_u64(scan_n, kScanTile) + 1) * 4);
    L.bytes = off;
    int tb = bits_for(n_tiles);
    L.tile_passes = tb == 0 ? 0 : (tb + 7) / 8;
    return L;
}

// ------------------------------------------------------------------ device helpers
// Hint: fetch the line holding p into L2 (no value returned, no fault).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Float32 camera depth with a fixed operation order (no contraction).
__device__ __forceinline__ float depth32(const float *vm, float x, float y, float z) {
    float s = __fadd_rn(__fmul_rn(vm[8], x), __fmul_rn(vm[9], y));
    s = __fadd_rn(s, __fmul_rn(vm[10], z));
    return __fadd_rn(s, vm[11]);
}

// Q(X, Y) = a X^2 + 2 b X Y + c Y^2 in a fixed unfused order (binning decisions).
__device__ __forceinline__ float quad_rn(float a, float b2, float c, float X, float Y) {
    float t1 = __fmul_rn(__fmul_rn(a, X), X);
    float t2 = __fmul_rn(__fmul_rn(b2, X), Y);
    float t3 = __fmul_rn(__fmul_rn(c, Y), Y);
    return __fadd_rn(__fadd_rn(t1, t2), t3);
}

// Minimum of Q over the rectangle of pixel centres [px0..px1] x [py0..py1],
// compared with qm. Q is convex: 0 if the rectangle holds the centre, else the
// minimum lies on an edge at the clamped 1-D minimiser.
// ia, ic are the correctly rounded reciprocals 1/a, 1/c.
__device__ __forceinline__ bool tile_hit(float u, float v, float a, float b, float c, float ia, float ic, float qm,
                                         int px0, int px1, int py0, int py1) {
    const float X0 = __fsub_rn(__fadd_rn((float)px0, 0.5f), u);
    const float X1 = __fsub_rn(__fadd_rn((float)px1, 0.5f), u);
    const float Y0 = __fsub_rn(__fadd_rn((float)py0, 0.5f), v);
    const float Y1 = __fsub_rn(__fadd_rn((float)py1, 0.5f), v);
    if (X0 <= 0.f && 0.f <= X1 && Y0 <= 0.f && 0.f <= Y1) return true;
    const float b2 = __fadd_rn(b, b);
    float best = __int_as_float(0x7f800000);
    {
        float ys = __fmul_rn(-__fmul_rn(b, X0), ic);
        ys = fminf(fmaxf(ys, Y0), Y1);
        best = fminf(best, quad_rn(a, b2, c, X0, ys));
        ys = __fmul_rn(-__fmul_rn(b, X1), ic);
        ys = fminf(fmaxf(ys, Y0), Y1);
        best = fminf(best, quad_rn(a, b2, c, X1, ys));
    }
    {
        float xs = __fmul_rn(-__fmul_rn(b, Y0), ia);
        xs = fminf(fmaxf(xs, X0), X1);
        best = fminf(best, quad_rn(a, b2, c, xs, Y0));
        xs = __fmul_rn(-__fmul_rn(b, Y1), ia);
        xs = fminf(fmaxf(xs, X0), X1);
        best = fminf(best, quad_rn(a, b2, c, xs, Y1));
    }
    return best <= qm;
}

// Pixel box of a splat: x in [ceil(u - ext_x - 1/2), floor(u + ext_x - 1/2)] clipped
// to the image (empty if x0 > x1), same in y.
__device__ __forceinline__ void pixel_box(float u, float v, float ext_x, float ext_y, int W, int H, int &x0,
                                          int &x1, int &y0, int &y1) {
    float fx0 = ceilf(__fsub_rn(__fsub_rn(u, ext_x), 0.5f));
    float fx1 = floorf(__fsub_rn(__fadd_rn(u, ext_x), 0.5f));
    float fy0 = ceilf(__fsub_rn(__fsub_rn(v, ext_y), 0.5f));
    float fy1 = floorf(__fsub_rn(__fadd_rn(v, ext_y), 0.5f));
    fx0 = fminf(fmaxf(fx0, 0.f), (float)W);
    fy0 = fminf(fmaxf(fy0, 0.f), (float)H);
    fx1 = fmaxf(fminf(fx1, (float)(W - 1)), -1.f);
    fy1 = fmaxf(fminf(fy1, (float)(H - 1)), -1.f);
    x0 = (int)fx0; x1 = (int)fx1; y0 = (int)fy0; y1 = (int)fy1;
}

// Screen-space evaluation of one (pixel, splat) pair, shared by forward and
// backward so that both take bit-identical decisions.
struct PairEval {
    float Q, lq, p, G, alpha_raw, alpha;  // lq = log2 Q
};

// Q = d^T C d of the pair (clamped at 0), d = (dx, dy), C the conic [a, b2/2; b2/2, c].
__device__ __forceinline__ float pair_q(float dx, float dy, float a, float b2, float c) {
    const float t = __fmaf_rn(a, dx, __fmul_rn(b2, dy));
    return fmaxf(__fmaf_rn(__fmul_rn(c, dy), dy, __fmul_rn(dx, t)), 0.f);
}

// p = Q^(beta/2) (Q = 0 gives 0), G = exp(-p/2), alpha = min(alpha_max, o G).
__device__ __forceinline__ void pair_alpha(float Q, float hb, float o, float alpha_max, PairEval &r) {
    const float lq = lg2_approx(Q);
    const float p = ex2_approx(__fmul_rn(hb, lq));
    const float G = ex2_approx(__fmul_rn(kNegHalfLog2e, p));
    const float ar = __fmul_rn(o, G);
    r.Q = Q; r.lq = lq; r.p = p; r.G = G; r.alpha_raw = ar; r.alpha = fminf(alpha_max, ar);
}

// Returns false if the pair is outside the support (Q > q_cut) or alpha < alpha_min. A lane
// outside the support skips the special-function work (r then holds Q only).
__device__ __forceinline__ bool eval_pair(float dx, float dy, float a, float b2, float c, float qcut, float hb,
                                          float o, float alpha_max, float alpha_min, PairEval &r) {
    const float Q = pair_q(dx, dy, a, b2, c);
    r.Q = Q;
    if (Q > qcut) return false;
    pair_alpha(Q, hb, o, alpha_max, r);
    return r.alpha >= alpha_min;
}

// The same decision and values without a branch: every lane does the special-function work and
// r is filled in full (outside the support p may be +inf and G, alpha 0; Q is finite or +inf,
// never NaN). For a loop whose body runs on every lane of the warp anyway, where the branch
// only adds divergence and reconvergence work.
__device__ __forceinline__ bool eval_pair_all(float dx, float dy, float a, float b2, float c, float qcut, float hb,
                                              float o, float alpha_max, float alpha_min, PairEval &r) {
    const float Q = pair_q(dx, dy, a, b2, c);
    pair_alpha(Q, hb, o, alpha_max, r);
    return Q <= qcut && r.alpha >= alpha_min;
}

// Real spherical harmonics up to degree 3 (Condon-Shortley phase, l-major,
// m = -l..l). Constants are sqrt2 K_l^|m| times the leading coefficient of
// P_l^|m| / sin^|m|, K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!):
//   l1: sqrt(3/4pi); l2: sqrt(15/4pi), sqrt(5/16pi), sqrt(15/16pi);
//   l3: sqrt(35/32pi), sqrt(105/4pi), sqrt(21/32pi), sqrt(7/16pi), sqrt(105/16pi).
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.48860251190291992f;
constexpr float kSH2a = 1.09254843059207907f;
constexpr float kSH2b = 0.31539156525252005f;
constexpr float kSH2c = 0.54627421529603959f;
constexpr float kSH3a = 0.59004358992664352f;
constexpr float kSH3b = 2.89061144264055405f;
constexpr float kSH3c = 0.45704579946446577f;
constexpr float kSH3d = 0.37317633259011546f;
constexpr float kSH3e = 1.44530572132027738f;

__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float *Y) {
    Y[0] = kSH0;
    if (deg < 1) return;
    Y[1] = -kSH1 * y; Y[2] = kSH1 * z; Y[3] = -kSH1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kSH2a * x * y; Y[5] = -kSH2a * y * z; Y[6] = kSH2b * (3.f * zz - 1.f);
    Y[7] = -kSH2a * x * z; Y[8] = kSH2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kSH3a * y * (3.f * xx - yy);
    Y[10] = kSH3b * x * y * z;
    Y[11] = -kSH3c * y * (5.f * zz - 1.f);
    Y[12] = kSH3d * z * (5.f * zz - 3.f);
    Y[13] = -kSH3c * x * (5.f * zz - 1.f);
    Y[14] = kSH3e * z * (xx - yy);
    Y[15] = -kSH3a * x * (xx - 3.f * yy);
}

// Gradient of each basis polynomial with respect to (x, y, z).
__device__ __forceinline__ void sh_grad(int deg, float x, float y, float z, float (*dY)[3]) {
    dY[0][0] = 0.f; dY[0][1] = 0.f; dY[0][2] = 0.f;
    if (deg < 1) return;
    dY[1][0] = 0.f; dY[1][1] = -kSH1; dY[1][2] = 0.f;
    dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = kSH1;
    dY[3][0] = -kSH1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    if (deg < 2) return;
    dY[4][0] = kSH2a * y; dY[4][1] = kSH2a * x; dY[4][2] = 0.f;
    dY[5][0] = 0.f; dY[5][1] = -kSH2a * z; dY[5][2] = -kSH2a * y;
    dY[6][0] = 0.f; dY[6][1] = 0.f; dY[6][2] = 6.f * kSH2b * z;
    dY[7][0] = -kSH2a * z; dY[7][1] = 0.f; dY[7][2] = -kSH2a * x;
    dY[8][0] = 2.f * kSH2c * x; dY[8][1] = -2.f * kSH2c * y; dY[8][2] = 0.f;
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    dY[9][0] = -6.f * kSH3a * x * y; dY[9][1] = -3.f * kSH3a * (xx - yy); dY[9][2] = 0.f;
    dY[10][0] = kSH3b * y * z; dY[10][1] = kSH3b * x * z; dY[10][2] = kSH3b * x * y;
    dY[11][0] = 0.f; dY[11][1] = -kSH3c * (5.f * zz - 1.f); dY[11][2] = -10.f * kSH3c * y * z;
    dY[12][0] = 0.f; dY[12][1] = 0.f; dY[12][2] = kSH3d * (15.f * zz - 3.f);
    dY[13][0] = -kSH3c * (5.f * zz - 1.f); dY[13][1] = 0.f; dY[13][2] = -10.f * kSH3c * x * z;
    dY[14][0] = 2.f * kSH3e * x * z; dY[14][1] = -2.f * kSH3e * y * z; dY[14][2] = kSH3e * (xx - yy);
    dY[15][0] = -3.f * kSH3a * (xx - yy); dY[15][1] = 6.f * kSH3a * x * y; dY[15][2] = 0.f;
}

// Gradient of sum_k al[k] Y_k with respect to (x, y, z), accumulated into g
// without forming the per-basis gradients (same polynomials as sh_grad).
__device__ __forceinline__ void sh_grad_dot(int deg, float x, float y, float z, const float *al, float &gx,
                                            float &gy, float &gz) {
    gx = 0.f; gy = 0.f; gz = 0.f;
    if (deg < 1) return;
    gy -= kSH1 * al[1]; gz += kSH1 * al[2]; gx -= kSH1 * al[3];
    if (deg < 2) return;
    gx += kSH2a * (y * al[4] - z * al[7]) + 2.f * kSH2c * x * al[8];
    gy += kSH2a * (x * al[4] - z * al[5]) - 2.f * kSH2c * y * al[8];
    gz += -kSH2a * (y * al[5] + x * al[7]) + 6.f * kSH2b * z * al[6];
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += -6.f * kSH3a * x * y * al[9] + kSH3b * y * z * al[10] - kSH3c * (5.f * zz - 1.f) * al[13] +
          2.f * kSH3e * x * z * al[14] - 3.f * kSH3a * (xx - yy) * al[15];
    gy += -3.f * kSH3a * (xx - yy) * al[9] + kSH3b * x * z * al[10] - kSH3c * (5.f * zz - 1.f) * al[11] -
          2.f * kSH3e * y * z * al[14] + 6.f * kSH3a * x * y * al[15];
    gz += kSH3b * x * y * al[10] - 10.f * kSH3c * y * z * al[11] + kSH3d * (15.f * zz - 3.f) * al[12] -
          10.f * kSH3c * x * z * al[13] + kSH3e * (xx - yy) * al[14];
}

// phi(beta) of Eq. 7 by reading mode, and d phi / d beta.
__device__ __forceinline__ float phi_beta(float beta, float rho, int mode, float &dphi) {
    if (mode == 0) { dphi = 0.f; return 1.f; }
    const float k = (mode == 1) ? rho : (rho - 2.f);
    const float arg = (mode == 1) ? rho * (beta - 2.f) : k * beta;
    const float s = 1.f / (1.f + expf(-arg));
    dphi = 2.f * k * s * (1.f - s);
    return 2.f * s;
}

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float *R) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

__device__ __forceinline__ void set_error(uint32_t *err, uint32_t bit) {
    if ((*(volatile uint32_t *)err & bit) == 0) atomicOr(err, bit);
}


// ------------------------------------------------------------------ kernel arguments
struct PreArgs {
    int n;
    int first, count;  // the splats [first, first + count) of the n
    const float4 *pos_op, *lsb, *quat;
    const void *color;  // Params::color_storage
    float4 *rec;     // [nV][4]
    uint4 *binrec;   // [nV][2]
    unsigned long long *total;
    uint32_t *err;
    Params P;
    ViewSet V;
};

struct PreBwdArgs {
    int n;
    int first, count;  // the splats [first, first + count) of the n
    const float4 *pos_op, *lsb, *quat;
    const void *color;  // Params::color_storage
    const float4 *rec;
    const float4 *g2d;  // [nV][4]
    float4 *g_pos_op, *g_lsb, *g_quat;
    float *g_color;
    Params P;
    ViewSet V;
};

struct EmitArgs {
    uint32_t n_entries;
    int n;  // splats per view
    const uint4 *rinfo;        // per rank: entry, hit mask, key of the box's first tile, box width | tiles_x << 6
    const uint32_t *offsets;   // exclusive scan of tiles touched in that order
    const float4 *rec;
    const uint4 *binrec;
    const unsigned long long *total;  // instances found by the preprocess
    uint32_t *ikey, *ival;
    uint64_t cap;
    uint32_t *err;
    ViewSet V;
};

struct BinArgs {
    int n, n_views;
    uint32_t n_entries;
    const float4 *rec;
    const uint4 *binrec;
    const unsigned long long *total;
    uint32_t *err;
    // bins
    uint32_t *header;  // [0] n_inst
    uint32_t *dkey[2], *dval[2], *rcount, *ikey[2], *ival[2];
    uint4 *rinfo;
    uint2 *ranges;
    uint32_t *queue;
    uint32_t *hist, *partials;
    uint64_t cap;
    int tile_bits;
    bool build_queue;
    ViewSet V;
};

struct FwdArgs {
    const float4 *rec;
    const uint32_t *inst_entry;
    const uint2 *ranges;
    const uint32_t *queue;  // NULL: one CTA per tile
    uint32_t *counter;
    float *color, *depth, *alpha, *normal, *t_final;
    uint32_t *last, *n_contrib, *n_eval;
    unsigned long long *n_events;  // with n_eval: (warp block, splat) pairs passing the warp cull
    uint32_t n_entries;            // (view, splat) entries: the bound of every listed entry
    uint32_t *err;                 // error word (debug-build bounds checks)
    int batch;
    float alpha_min, alpha_max, t_min;
    float bg[3];
    ViewSet V;
};

struct BwdArgs {
    const float4 *rec;
    const uint32_t *inst_entry;
    const uint2 *ranges;
    const uint32_t *queue;
    uint32_t *counter;
    const float *color, *depth, *normal, *t_final;
    const uint32_t *last;
    const float *g_color, *g_depth, *g_alpha, *g_normal;
    float *g2d;
    uint32_t n_entries;  // (view, splat) entries: the bound of every listed entry
    uint32_t *err;       // error word (debug-build bounds checks)
    int batch;
    float alpha_min, alpha_max;
    ViewSet V;
};

// ------------------------------------------------------------------ launchers
cudaError_t launch_preprocess(const PreArgs &a, cudaStream_t s);
cudaError_t launch_preprocess_bwd(const PreBwdArgs &a, cudaStream_t s);
cudaError_t launch_bin(const BinArgs &a, cudaStream_t s);
// Stable LSD radix sort of (key, value) pairs on bits [0, bits), 8 bits a pass (binning.cu).
cudaError_t radix_sort(uint32_t *keys[2], uint32_t *vals[2], bool iota_vals, const uint32_t *n_dev,
                       uint32_t n_host_max, int bits, uint32_t *hist, uint32_t *partials, cudaStream_t s);
cudaError_t launch_render_fwd(const FwdArgs &a, cudaStream_t s);
cudaError_t launch_render_bwd(const BwdArgs &a, cudaStream_t s);
bool tile_shape_supported(int tw, int th);

}  // namespace ges
