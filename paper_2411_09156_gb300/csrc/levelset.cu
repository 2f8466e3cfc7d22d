// Level-set points from rendered depth (Sec. 3.3, "Mesh Extraction"; level alpha = 0.3,
// Sec. 4.2): for each sampled pixel, the point x0 on its ray at the rendered depth,
// the 16 splat centres nearest to x0, the density of Eq. 9 marched over
// [-3 sigma_g(v), 3 sigma_g(v)] along the ray, the first upward crossing of the level
// by linear interpolation, and the normal grad f / |grad f| there.
//
// k_ls_start places x0 (depth D / A along the pixel ray); the KNN point queries of
// knn.cu (taken in grid-cell order) find the 16 nearest centres; k_ls_march, one thread per
// pixel, turns each neighbour into the ray form of its axis coordinates,
// loc_k(t) = loc_k(x0) + t loc_k(v), so a sample costs three fused multiply-adds per axis and
// the falloff; densities of 16 samples at a time are held in registers and the march stops
// after the chunk holding the first crossing.
#include <cstring>

#include "ges_internal.cuh"
#include "splat_rec.cuh"

namespace ges {

size_t knn_points_workspace(int32_t n, int32_t m);
cudaError_t knn_points_run(int32_t n, const float4 *pos, int32_t m, const float4 *pts, void *workspace,
                           int32_t *knn, cudaStream_t s);

namespace {

constexpr int kK = GES_KNN_K;
// one warp per CTA: marches differ in length, and a CTA of several warps would hold its slot
// until its longest march ended
constexpr int kLsThreads = 32;
constexpr int kLsChunk = 16;  // march samples whose densities a thread holds at once
constexpr float kHalfLog2e = 0.72134752044448170f;

struct LsArgs {
    int n, m, n_views, n_steps;
    float level, rho;
    int phi_mode;
    const float4 *pos_op, *lsb, *quat;
    int width[kMaxViews], height[kMaxViews];
    long long pix_base[kMaxViews];
    float fx[kMaxViews], fy[kMaxViews], cx[kMaxViews], cy[kMaxViews];
    float vm[kMaxViews][12];
    const float *depth, *alpha;
    const int32_t *pixels;  // [m][2]: view, pixel index y * W + x
    float4 *pts;            // [m]: x0, valid
    float4 *rec;            // [n][kRec]
    const int32_t *knn;     // [m][16]
    float *out;             // [m][8]
};

// Camera-frame ray (X/Z, Y/Z, 1) of pixel `pix` of view v, and its unit world direction.
__device__ __forceinline__ void pixel_ray(const LsArgs &a, int v, int pix, float *rc, float *dir) {
    const int W = a.width[v];
    const int px = pix % W, py = pix / W;
    rc[0] = ((float)px + 0.5f - a.cx[v]) / a.fx[v];
    rc[1] = ((float)py + 0.5f - a.cy[v]) / a.fy[v];
    rc[2] = 1.f;
    const float *m = a.vm[v];
    float d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) d[c] = m[c] * rc[0] + m[4 + c] * rc[1] + m[8 + c] * rc[2];  // R^T rc
    const float inv = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    dir[0] = d[0] * inv; dir[1] = d[1] * inv; dir[2] = d[2] * inv;
}

__global__ void __launch_bounds__(256) k_ls_start(LsArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.m) return;
    const int v = a.pixels[2 * (size_t)k], pix = a.pixels[2 * (size_t)k + 1];
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (v >= 0 && v < a.n_views && pix >= 0 && (long long)pix < (long long)a.width[v] * a.height[v]) {
        const float D = a.depth[a.pix_base[v] + pix], A = a.alpha[a.pix_base[v] + pix];
        if (A >= 1e-4f && isfinite(D)) {
            float rc[3], dir[3];
            pixel_ray(a, v, pix, rc, dir);
            const float z = D / A;
            const float *m = a.vm[v];
            // x0 = c + R^T (rc z), c = -R^T t
            float x[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                x[c] = m[c] * (rc[0] * z - m[3]) + m[4 + c] * (rc[1] * z - m[7]) + m[8 + c] * (rc[2] * z - m[11]);
            if (isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2])) p = make_float4(x[0], x[1], x[2], 1.f);
        }
    }
    a.pts[k] = p;
}

__global__ void __launch_bounds__(256) k_ls_prep(LsArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) build_splat_rec(a.pos_op, a.quat, a.lsb, a.rho, a.phi_mode, i, a.rec);
}

// Neighbour s of a pixel in ray form: its axis coordinates over s' at x0 (l0) and along the
// ray direction (lv), so that loc(t) = l0 + t lv; plus opacity and beta / 2.
struct RayTerm {
    float l0[3], lv[3], o, hb;
};

__device__ __forceinline__ RayTerm ray_term(const NbRec &N, float4 p0, const float *dir) {
    const float dx = p0.x - N.r0.x, dy = p0.y - N.r0.y, dz = p0.z - N.r0.z;
    RayTerm r;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float is = sqrtf(N.ia[c]);  // 1 / s'
        r.l0[c] = (N.R[c] * dx + N.R[3 + c] * dy + N.R[6 + c] * dz) * is;
        r.lv[c] = (N.R[c] * dir[0] + N.R[3 + c] * dir[1] + N.R[6 + c] * dir[2]) * is;
    }
    r.o = N.r0.w;
    r.hb = 0.5f * N.beta;
    return r;
}

// o exp(-1/2 Q^(beta/2)) at loc(t), with the hardware base-2 approximations (flushing
// subnormals: Q below 2^-126 counts as 0, where the term is o).
__device__ __forceinline__ float term_at(const RayTerm &r, float t) {
    const float l0 = fmaf(t, r.lv[0], r.l0[0]), l1 = fmaf(t, r.lv[1], r.l0[1]), l2 = fmaf(t, r.lv[2], r.l0[2]);
    const float Q = fmaf(l0, l0, fmaf(l1, l1, l2 * l2));
    return r.o * ex2_approx(-kHalfLog2e * ex2_approx(r.hb * lg2_approx(Q)));
}

// One thread per pixel. The samples are taken kLsChunk at a time: each neighbour is put in
// ray form once per chunk and its terms added to the chunk's densities in registers, then
// the chunk is scanned for the first upward crossing (so nothing is staged in shared memory).
__global__ void __launch_bounds__(kLsThreads) k_ls_march(LsArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.m) return;
    float *o8 = a.out + 8 * (size_t)k;
    const float4 p0 = a.pts[k];
    if (p0.w == 0.f) {
#pragma unroll
        for (int q = 0; q < 8; ++q) o8[q] = 0.f;
        return;
    }
    const int v = a.pixels[2 * (size_t)k], pix = a.pixels[2 * (size_t)k + 1];
    float rc[3], dir[3];
    pixel_ray(a, v, pix, rc, dir);
    const int32_t *nb = a.knn + (size_t)k * kK;
    // neighbour s of this pixel, or -1 (lists are re-read from L1 rather than kept in an array)
    auto nbr = [&](int s) {
        const int i = __ldg(nb + s);
        return (i >= 0 && i < a.n) ? i : -1;
    };
    // g = the smallest exponent at x0, sigma_g(v)^2 = sum_k (r_k . v)^2 s'_k^2
    float pmin = __int_as_float(0x7f800000), sig2 = 0.f;
    for (int s = 0; s < kK; ++s) {
        const int i = nbr(s);
        if (i < 0) continue;
        const NbRec N = load_rec(a.rec, i);
        const float dx = p0.x - N.r0.x, dy = p0.y - N.r0.y, dz = p0.z - N.r0.z;
        float Q = 0.f, sv = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float is = sqrtf(N.ia[c]);  // 1 / s'
            const float pr = (N.R[c] * dx + N.R[3 + c] * dy + N.R[6 + c] * dz) * is;
            const float vr = N.R[c] * dir[0] + N.R[3 + c] * dir[1] + N.R[6 + c] * dir[2];
            Q = fmaf(pr, pr, Q);
            sv = fmaf(vr * vr, 1.f / N.ia[c], sv);
        }
        const float P = exp2f(0.5f * N.beta * log2f(Q));
        if (P < pmin) { pmin = P; sig2 = sv; }
    }
    const float sigma = sqrtf(sig2);
    const int ns = a.n_steps;
    const float dt = 6.f * sigma / (float)(ns - 1);
    float tprev = 0.f, dprev = 0.f, tstar = 0.f;
    bool found = false;
    for (int j0 = 0; j0 < ns && !found; j0 += kLsChunk) {
        float d[kLsChunk];
#pragma unroll
        for (int j = 0; j < kLsChunk; ++j) d[j] = 0.f;
        for (int s = 0; s < kK; ++s) {
            const int i = nbr(s);
            if (i < 0) continue;
            const RayTerm r = ray_term(load_rec(a.rec, i), p0, dir);
#pragma unroll
            for (int j = 0; j < kLsChunk; ++j) d[j] += term_at(r, fmaf((float)(j0 + j), dt, -3.f * sigma));
        }
#pragma unroll
        for (int j = 0; j < kLsChunk; ++j) {
            if (found || j0 + j >= ns) continue;
            const float t = fmaf((float)(j0 + j), dt, -3.f * sigma);
            if (j0 + j > 0 && dprev < a.level && a.level <= d[j]) {
                tstar = tprev + (a.level - dprev) / (d[j] - dprev) * (t - tprev);
                found = true;
            }
            tprev = t;
            dprev = d[j];
        }
    }
    if (!found) {
#pragma unroll
        for (int q = 0; q < 8; ++q) o8[q] = 0.f;
        return;
    }
    // normal: the direction of -grad d = sum_i t_i (beta_i/2) Q_i^(beta_i/2 - 1) Sigma_i^-1 (x - mu_i),
    // summed relative to its largest term (rescaled whenever a smaller exponent appears)
    float wx = 0.f, wy = 0.f, wz = 0.f;
    float pm = __int_as_float(0x7f800000);
    for (int s = 0; s < kK; ++s) {
        const int i = nbr(s);
        if (i < 0) continue;
        const NbRec N = load_rec(a.rec, i);
        const RayTerm r = ray_term(N, p0, dir);
        const float l[3] = {fmaf(tstar, r.lv[0], r.l0[0]), fmaf(tstar, r.lv[1], r.l0[1]),
                            fmaf(tstar, r.lv[2], r.l0[2])};
        const float Q = fmaf(l[0], l[0], fmaf(l[1], l[1], l[2] * l[2]));
        const float P = exp2f(r.hb * log2f(Q));
        if (P < pm) {
            const float scl = exp2f(-kHalfLog2e * (pm - P));
            if (pm != __int_as_float(0x7f800000)) { wx *= scl; wy *= scl; wz *= scl; }
            pm = P;
        }
        const float ct = Q > 0.f ? r.o * exp2f(-kHalfLog2e * (P - pm)) * r.hb * P / Q : 0.f;
        // Sigma^-1 (x - mu) = R diag(1 / s') loc
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float a_c = ct * l[c] * sqrtf(N.ia[c]);
            wx = fmaf(a_c, N.R[c], wx);
            wy = fmaf(a_c, N.R[3 + c], wy);
            wz = fmaf(a_c, N.R[6 + c], wz);
        }
    }
    const float wn = sqrtf(wx * wx + wy * wy + wz * wz);
    const float iw = wn > 0.f ? 1.f / wn : 0.f;
    o8[0] = p0.x + tstar * dir[0];
    o8[1] = p0.y + tstar * dir[1];
    o8[2] = p0.z + tstar * dir[2];
    o8[3] = wx * iw;
    o8[4] = wy * iw;
    o8[5] = wz * iw;
    o8[6] = tstar;
    o8[7] = wn > 0.f ? 1.f : 0.f;
}

struct LsLayout {
    uint64_t knn_ws, rec, pts, lists, bytes;
};

inline uint64_t al256l(uint64_t x) { return (x + 255) & ~uint64_t(255); }

LsLayout ls_layout(int32_t n, int32_t m) {
    LsLayout L;
    uint64_t off = 0;
    L.knn_ws = off; off = al256l(off + knn_points_workspace(n, m));
    L.rec = off; off = al256l(off + 16ull * kRec * n);
    L.pts = off; off = al256l(off + 16ull * m);
    L.lists = off; off = al256l(off + 4ull * kK * m);
    L.bytes = off;
    return L;
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" size_t ges_levelset_workspace_bytes(int32_t n, int32_t m) {
    if (n < GES_KNN_K || (uint64_t)n > (1ull << 26) || m < 1 || (uint64_t)m > (1ull << 28)) return 0;
    return ls_layout(n, m).bytes;
}

extern "C" ges_status ges_levelset(int32_t n, const float *pos_op, const float *lscale_beta, const float *quat,
                                   const ges_config *cfg, int32_t n_views, const ges_camera *cams, const float *depth,
                                   const float *alpha, int32_t m, const int32_t *pixels, int32_t n_steps, float level,
                                   void *workspace, size_t workspace_bytes, float *points, void *stream) {
    GES_RANGE();
    if (n < GES_KNN_K || (uint64_t)n > (1ull << 26) || m < 1 || (uint64_t)m > (1ull << 28)) return GES_ERR_INVALID_ARG;
    if (!pos_op || !lscale_beta || !quat || !cfg || !cams || !depth || !alpha || !pixels || !workspace || !points)
        return GES_ERR_INVALID_ARG;
    if (n_views < 1 || n_views > kMaxViews || n_steps < 2 || n_steps > 1024 || !(level > 0.f) || !isfinite(level))
        return GES_ERR_INVALID_ARG;
    if (((uintptr_t)pos_op | (uintptr_t)lscale_beta | (uintptr_t)quat) & 15u) return GES_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) || cfg->phi_mode < 0 || cfg->phi_mode > 2 || !isfinite(cfg->rho))
        return GES_ERR_INVALID_ARG;
    const LsLayout L = ls_layout(n, m);
    if (workspace_bytes < L.bytes) return GES_ERR_INVALID_ARG;
    LsArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n; a.m = m; a.n_views = n_views; a.n_steps = n_steps; a.level = level;
    a.rho = cfg->rho; a.phi_mode = cfg->phi_mode;
    a.pos_op = reinterpret_cast<const float4 *>(pos_op);
    a.lsb = reinterpret_cast<const float4 *>(lscale_beta);
    a.quat = reinterpret_cast<const float4 *>(quat);
    long long pb = 0;
    for (int v = 0; v < n_views; ++v) {
        const ges_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > (1 << 15) || c.height > (1 << 15) || !(c.fx > 0.f) ||
            !(c.fy > 0.f))
            return GES_ERR_INVALID_ARG;
        a.width[v] = c.width; a.height[v] = c.height; a.pix_base[v] = pb;
        a.fx[v] = c.fx; a.fy[v] = c.fy; a.cx[v] = c.cx; a.cy[v] = c.cy;
        for (int q = 0; q < 12; ++q) a.vm[v][q] = c.viewmat[q];
        pb += (long long)c.width * c.height;
    }
    a.depth = depth; a.alpha = alpha; a.pixels = pixels;
    char *ws = static_cast<char *>(workspace);
    a.pts = reinterpret_cast<float4 *>(ws + L.pts);
    a.rec = reinterpret_cast<float4 *>(ws + L.rec);
    int32_t *lists = reinterpret_cast<int32_t *>(ws + L.lists);
    a.knn = lists;
    a.out = points;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_ls_start<<<ceil_div_u64(m, 256), 256, 0, s>>>(a);
    k_ls_prep<<<ceil_div_u64(n, 256), 256, 0, s>>>(a);
    if (knn_points_run(n, a.pos_op, m, a.pts, ws + L.knn_ws, lists, s) != cudaSuccess) return GES_ERR_CUDA;
    k_ls_march<<<ceil_div_u64(m, kLsThreads), kLsThreads, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GES_OK : GES_ERR_CUDA;
}
