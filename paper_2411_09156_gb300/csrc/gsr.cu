// Generalized surface regularization (GSR) at sample points, Eq. 9-13 (Sec. 3.3):
// the density of the 16 nearest splats (Eq. 9), the ideal flat density of the
// dominant splat g* (Eq. 10), the SDFs of both (Eq. 11), L_sdf (Eq. 12) and L_nor
// (Eq. 13), forward and analytic backward.
//
// k_gsr_prep turns each splat into an 80-byte record (centre, opacity, rotation,
// 1/s'^2, beta, smallest scale and its axis index), so a sample evaluates a
// neighbour from one record: the Mahalanobis form is taken in the splat's own axes,
// Q = sum_k (r_k . delta)^2 / s'_k^2, with no cancellation for flat splats (whose
// inverse covariance spans 1e4 to 1e8 in float32). k_gsr_sample runs one thread per
// sample: the sample's offset o = R_j (s'_j * z) from its splat's centre, the
// neighbour sums d and w (the direction of -grad d, relative to its largest term),
// g*, the losses, and then (a second pass over the neighbours, recomputing the
// per-neighbour terms instead of holding 16 sets in registers) the gradient with
// respect to each neighbour's centre, opacity, rotation, scales and beta, g*'s
// centre, axis, smallest scale and beta, and splat j's centre, rotation and scales
// (through x), all added into a 17-float accumulator per splat in the splats' own
// frames: the scale gradient of a flat axis is formed from that axis' projections,
// never recovered from a world-frame matrix gradient, where it would be a 1e-4 part
// cancelled out of the in-plane terms. k_gsr_chain takes each accumulator through
// s' = phi(beta) exp(l) and R(q) to the log-scales, beta and quaternion.
#include <cstring>

#include "ges_internal.cuh"
#include "splat_rec.cuh"

namespace ges {
namespace {

constexpr int kK = GES_KNN_K;
constexpr int kAcc = 17;  // dL/d: mu (3), o, R (9, row-major), s' (3), beta
constexpr int kGsrThreads = 128;
constexpr float kDMin = 1e-30f;
constexpr float kLn2 = 0.69314718055994531f;
constexpr float kHalfLog2e = 0.72134752044448170f;  // exp(-x/2) = exp2(-kHalfLog2e x)

struct GsrArgs {
    int n, m;
    int phi_mode;
    float rho;
    const float4 *pos_op, *lsb, *quat;
    const int32_t *knn;
    const int32_t *sample_splat;
    const float *sample_z;
    float lambda_sdf, lambda_nor, inv_m;
    float4 *rec;        // [n][kRec]
    float *acc;         // [n][kAcc], NULL: forward only
    double *partial;    // [blocks][2]
    float *losses;      // [3]
    float *sample_out;  // [m][8] or NULL
    float4 *g_pos_op, *g_lsb, *g_quat;
};

__device__ __forceinline__ void splat_frame(const GsrArgs &a, int i, float *R, float *sp, float &dphi, float &phi,
                                            float *es, float &qinv, float *qn) {
    ges::splat_frame(a.quat, a.lsb, a.rho, a.phi_mode, i, R, sp, dphi, phi, es, qinv, qn);
}

__global__ void __launch_bounds__(256) k_gsr_prep(GsrArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    build_splat_rec(a.pos_op, a.quat, a.lsb, a.rho, a.phi_mode, i, a.rec);
    if (a.acc) {
#pragma unroll
        for (int q = 0; q < kAcc; ++q) a.acc[(size_t)i * kAcc + q] = 0.f;
    }
}

// Per-neighbour terms: delta = x - mu, v = A delta, Q = delta.v (as a sum over the
// axes), P = Q^(beta/2), G = exp(-P/2), t = o G. The weight of v in -grad d is
// t (beta/2) P / Q; relative to the largest term it is o exp(-(P - P_min)/2) (beta/2) P / Q.
struct NbTerms {
    float dx, dy, dz, vx, vy, vz, Q, lq, hb, P, G, t, o;
};

// (ox, oy, oz) is the sample's offset from the centre (cx, cy, cz) of the splat it was
// drawn from: delta = (centre - mu) + offset, so the sample's own splat sees its offset
// exactly and near neighbours a difference of nearby centres, which float32 represents
// without the cancellation of (centre + offset) - mu.
__device__ __forceinline__ NbTerms nb_terms(const NbRec &N, float cx, float cy, float cz, float ox, float oy,
                                           float oz) {
    NbTerms T;
    T.dx = (cx - N.r0.x) + ox; T.dy = (cy - N.r0.y) + oy; T.dz = (cz - N.r0.z) + oz;
    T.vx = T.vy = T.vz = 0.f;
    float Q = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float p = N.R[k] * T.dx + N.R[3 + k] * T.dy + N.R[6 + k] * T.dz;
        const float ap = p * N.ia[k];
        Q = fmaf(ap, p, Q);
        T.vx = fmaf(ap, N.R[k], T.vx);
        T.vy = fmaf(ap, N.R[3 + k], T.vy);
        T.vz = fmaf(ap, N.R[6 + k], T.vz);
    }
    T.Q = Q;
    T.hb = 0.5f * N.beta;
    T.lq = log2f(T.Q);  // -inf at Q = 0
    T.P = exp2f(T.hb * T.lq);
    T.G = exp2f(-kHalfLog2e * T.P);
    T.o = N.r0.w;
    T.t = T.o * T.G;
    return T;
}

__device__ __forceinline__ void red_add(float *p, float v) {
    if (v != 0.f) atomicAdd(p, v);
}

__global__ void __launch_bounds__(kGsrThreads) k_gsr_sample(GsrArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    float l_sdf = 0.f, l_nor = 0.f;
    if (k < a.m) {
        const int j = a.sample_splat[k];
        if (j >= 0 && j < a.n) {
            float R[9], sp[3], es[3], qn[4], dphi, phi, qinv;
            splat_frame(a, j, R, sp, dphi, phi, es, qinv, qn);
            const float z0 = a.sample_z[3 * (size_t)k], z1 = a.sample_z[3 * (size_t)k + 1],
                        z2 = a.sample_z[3 * (size_t)k + 2];
            const float4 pj = __ldg(a.pos_op + j);
            const float m0 = sp[0] * z0, m1 = sp[1] * z1, m2 = sp[2] * z2;
            const float ox = R[0] * m0 + R[1] * m1 + R[2] * m2;  // x - mu_j
            const float oy = R[3] * m0 + R[4] * m1 + R[5] * m2;
            const float oz = R[6] * m0 + R[7] * m1 + R[8] * m2;
            const int32_t *nb = a.knn + (size_t)j * kK;
            // forward: d, g* (the smallest exponent P, first on ties: the largest falloff
            // exp(-P/2), decided where the falloffs themselves underflow), and -grad d's
            // direction w as a sum relative to the largest term exp(-P_min/2), rescaled
            // whenever a smaller P appears
            float d = 0.f, wx = 0.f, wy = 0.f, wz = 0.f, pmin = __int_as_float(0x7f800000);
            int best = -1;
            for (int s = 0; s < kK; ++s) {
                const int i = __ldg(nb + s);
                if (i < 0 || i >= a.n) continue;
                const NbTerms T = nb_terms(load_rec(a.rec, i), pj.x, pj.y, pj.z, ox, oy, oz);
                d += T.t;
                if (T.P < pmin) {
                    if (best >= 0) {
                        const float sc = exp2f(-kHalfLog2e * (pmin - T.P));
                        wx *= sc; wy *= sc; wz *= sc;
                    }
                    pmin = T.P;
                    best = s;
                }
                const float ct = T.Q > 0.f ? T.o * exp2f(-kHalfLog2e * (T.P - pmin)) * T.hb * T.P / T.Q : 0.f;
                wx = fmaf(ct, T.vx, wx); wy = fmaf(ct, T.vy, wy); wz = fmaf(ct, T.vz, wz);
            }
            if (best >= 0) {
                const int gs = __ldg(nb + best);
                const NbRec S = load_rec(a.rec, gs);
                const float n0 = S.km == 0 ? S.R[0] : (S.km == 1 ? S.R[1] : S.R[2]);
                const float n1 = S.km == 0 ? S.R[3] : (S.km == 1 ? S.R[4] : S.R[5]);
                const float n2 = S.km == 0 ? S.R[6] : (S.km == 1 ? S.R[7] : S.R[8]);
                const float ex = (pj.x - S.r0.x) + ox, ey = (pj.y - S.r0.y) + oy, ez = (pj.z - S.r0.z) + oz;
                const float e_raw = ex * n0 + ey * n1 + ez * n2;
                const float sg = e_raw < 0.f ? -1.f : 1.f;
                const float e = sg * e_raw;
                const float nsx = sg * n0, nsy = sg * n1, nsz = sg * n2;
                const float smin = S.smin, hs = 0.5f * S.beta;
                const float fbar = e > 0.f ? smin * exp2f(hs * log2f(e / smin)) : 0.f;
                const float dc = fminf(fmaxf(d, kDMin), 1.f);
                const float pl = -2.f * logf(dc);
                const float f = pl > 0.f ? smin * sqrtf(pl) : 0.f;
                const float wn = sqrtf(wx * wx + wy * wy + wz * wz);
                const float iw = wn > 0.f ? 1.f / wn : 0.f;
                const float ux = wx * iw, uy = wy * iw, uz = wz * iw;
                const float qx = ux - nsx, qy = uy - nsy, qz = uz - nsz;
                l_sdf = fabsf(fbar - f);
                l_nor = qx * qx + qy * qy + qz * qz;
                if (a.sample_out) {
                    float *o = a.sample_out + 8 * (size_t)k;
                    o[0] = pj.x + ox; o[1] = pj.y + oy; o[2] = pj.z + oz; o[3] = d; o[4] = f; o[5] = fbar;
                    o[6] = ux * nsx + uy * nsy + uz * nsz;
                    o[7] = (float)best;
                }
                if (a.acc) {
                    const float gL = a.inv_m;
                    const float gfb = a.lambda_sdf * gL * (fbar > f ? 1.f : (fbar < f ? -1.f : 0.f));
                    const float gf = -gfb;
                    // L_nor = |u - n*|^2
                    const float gux = 2.f * a.lambda_nor * gL * qx, guy = 2.f * a.lambda_nor * gL * qy,
                                guz = 2.f * a.lambda_nor * gL * qz;
                    const float gnsx = -gux, gnsy = -guy, gnsz = -guz;
                    const float gud = gux * ux + guy * uy + guz * uz;
                    const float gwx = (gux - gud * ux) * iw, gwy = (guy - gud * uy) * iw, gwz = (guz - gud * uz) * iw;
                    // fbar = s_min^(1 - hs) e^hs
                    float ge = 0.f, gsmin = 0.f, gbs = 0.f;
                    if (e > 0.f && smin > 0.f) {
                        ge = gfb * hs * fbar / e;
                        gsmin = gfb * (1.f - hs) * fbar / smin;
                        gbs = 0.5f * gfb * fbar * logf(e / smin);
                    }
                    // f = s_min sqrt(-2 ln d)
                    float gd = 0.f;
                    if (pl > 0.f && d > kDMin) {
                        gsmin += gf * f / smin;
                        gd = -gf * smin / (d * sqrtf(pl));
                    }
                    // e = sg (x - mu*) . n_raw, n* = sg n_raw; n_raw is column km of R*,
                    // s_min is s'*[km]
                    float gxx = ge * nsx, gxy = ge * nsy, gxz = ge * nsz;
                    float *ag = a.acc + (size_t)gs * kAcc;
                    red_add(ag + 0, -ge * nsx); red_add(ag + 1, -ge * nsy); red_add(ag + 2, -ge * nsz);
                    red_add(ag + 4 + S.km, sg * (ge * ex + gnsx));
                    red_add(ag + 7 + S.km, sg * (ge * ey + gnsy));
                    red_add(ag + 10 + S.km, sg * (ge * ez + gnsz));
                    red_add(ag + 13 + S.km, gsmin);
                    red_add(ag + 16, gbs);
                    // neighbours: d = sum t_i (unscaled), w = sum ct_i v_i (relative weights)
                    for (int s = 0; s < kK; ++s) {
                        const int i = __ldg(nb + s);
                        if (i < 0 || i >= a.n) continue;
                        const NbRec N = load_rec(a.rec, i);
                        const NbTerms T = nb_terms(N, pj.x, pj.y, pj.z, ox, oy, oz);
                        const float iq = T.Q > 0.f ? 1.f / T.Q : 0.f;
                        const float er = exp2f(-kHalfLog2e * (T.P - pmin));
                        const float ct = T.o * er * T.hb * T.P * iq;  // relative weight of v in w
                        const float gc = gwx * T.vx + gwy * T.vy + gwz * T.vz;
                        const float gvx = ct * gwx, gvy = ct * gwy, gvz = ct * gwz;
                        const float lnq = T.Q > 0.f ? T.lq * kLn2 : 0.f;
                        // the density path (t = o G) and the direction path (ct)
                        const float go = gd * T.G + gc * er * T.hb * T.P * iq;
                        const float gQ = -0.5f * gd * T.t * T.hb * T.P * iq +
                                         gc * ct * ((T.hb - 1.f) * iq - 0.5f * T.hb * T.P * iq);
                        const float ghb = -0.5f * gd * T.t * T.P * lnq +
                                          gc * ct * ((T.hb > 0.f ? 1.f / T.hb : 0.f) + lnq - 0.5f * T.P * lnq);
                        // Q = sum_k a_k p_k^2 and v = sum_k a_k p_k r_k with p_k = r_k . delta,
                        // a_k = 1/s'_k^2: per axis h_k = 2 gQ a_k p_k + a_k (r_k . g_v);
                        // dL/ddelta = sum_k h_k r_k, dL/dr_k = h_k delta + a_k p_k g_v,
                        // dL/da_k = gQ p_k^2 + p_k (r_k . g_v)
                        float gdx = 0.f, gdy = 0.f, gdz = 0.f;
                        float *ai = a.acc + (size_t)i * kAcc;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float r0c = N.R[c], r1c = N.R[3 + c], r2c = N.R[6 + c], ak = N.ia[c];
                            const float pk = r0c * T.dx + r1c * T.dy + r2c * T.dz;
                            const float gk = r0c * gvx + r1c * gvy + r2c * gvz;
                            const float hk = 2.f * gQ * ak * pk + ak * gk;
                            gdx = fmaf(hk, r0c, gdx); gdy = fmaf(hk, r1c, gdy); gdz = fmaf(hk, r2c, gdz);
                            const float apk = ak * pk;
                            red_add(ai + 4 + c, hk * T.dx + apk * gvx);
                            red_add(ai + 7 + c, hk * T.dy + apk * gvy);
                            red_add(ai + 10 + c, hk * T.dz + apk * gvz);
                            const float gak = gQ * pk * pk + pk * gk;
                            red_add(ai + 13 + c, gak * (-2.f * ak * sqrtf(ak)));  // da/ds' = -2 / s'^3
                        }
                        gxx += gdx; gxy += gdy; gxz += gdz;
                        red_add(ai + 0, -gdx); red_add(ai + 1, -gdy); red_add(ai + 2, -gdz);
                        red_add(ai + 3, go);
                        red_add(ai + 16, 0.5f * ghb);
                    }
                    // x = mu_j + R diag(s') z
                    float *aj = a.acc + (size_t)j * kAcc;
                    red_add(aj + 0, gxx); red_add(aj + 1, gxy); red_add(aj + 2, gxz);
                    const float gxv[3] = {gxx, gxy, gxz}, zv[3] = {z0, z1, z2};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
#pragma unroll
                        for (int r = 0; r < 3; ++r) red_add(aj + 4 + 3 * r + c, gxv[r] * zv[c] * sp[c]);
                        red_add(aj + 13 + c, zv[c] * (R[c] * gxx + R[3 + c] * gxy + R[6 + c] * gxz));
                    }
                }
            }
        }
    }
    // CTA sums of the two loss terms (double), in a fixed order
    __shared__ double s_red[2][kGsrThreads / 32];
    double d0 = l_sdf, d1 = l_nor;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d0 += __shfl_down_sync(0xffffffffu, d0, o);
        d1 += __shfl_down_sync(0xffffffffu, d1, o);
    }
    if ((threadIdx.x & 31) == 0) { s_red[0][threadIdx.x >> 5] = d0; s_red[1][threadIdx.x >> 5] = d1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < kGsrThreads / 32; ++w) { t0 += s_red[0][w]; t1 += s_red[1][w]; }
        a.partial[2 * (size_t)blockIdx.x] = t0;
        a.partial[2 * (size_t)blockIdx.x + 1] = t1;
    }
}

__global__ void __launch_bounds__(256) k_gsr_finalize(GsrArgs a, int nblocks) {
    __shared__ double s0[256], s1[256];
    const int t = threadIdx.x;
    double x0 = 0.0, x1 = 0.0;
    for (int b = t; b < nblocks; b += 256) {
        x0 += a.partial[2 * (size_t)b];
        x1 += a.partial[2 * (size_t)b + 1];
    }
    s0[t] = x0;
    s1[t] = x1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) { s0[t] += s0[t + o]; s1[t] += s1[t + o]; }
        __syncthreads();
    }
    if (t == 0) {
        const double m = (double)a.m;
        a.losses[0] = (float)(s0[0] / m);
        a.losses[1] = (float)(s1[0] / m);
        a.losses[2] = (float)((double)a.lambda_sdf * s0[0] / m + (double)a.lambda_nor * s1[0] / m);
    }
}

// Accumulated gradients of (mu, o, R, s', beta) -> (pos_op, lscale_beta, quat).
__global__ void __launch_bounds__(256) k_gsr_chain(GsrArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    float R[9], sp[3], es[3], qn[4], dphi, phi, qinv;
    splat_frame(a, i, R, sp, dphi, phi, es, qinv, qn);
    const float *g = a.acc + (size_t)i * kAcc;
    a.g_pos_op[i] = make_float4(g[0], g[1], g[2], g[3]);
    float GR[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) GR[q] = g[4 + q];
    // s' = phi(beta) exp(l)
    float gbeta = g[16];
    float gl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        gl[c] = g[13 + c] * sp[c];
        gbeta += g[13 + c] * dphi * es[c];
    }
    a.g_lsb[i] = make_float4(gl[0], gl[1], gl[2], gbeta);
    // R(q) -> unit quaternion -> quaternion
    const float w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    const float gw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
    const float gx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] -
                            2.f * x * GR[8]);
    const float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] -
                            2.f * y * GR[8]);
    const float gz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] +
                            x * GR[6] + y * GR[7]);
    const float dq = gw * w + gx * x + gy * y + gz * z;
    a.g_quat[i] = make_float4((gw - w * dq) * qinv, (gx - x * dq) * qinv, (gy - y * dq) * qinv, (gz - z * dq) * qinv);
}

struct GsrLayout {
    uint64_t rec, acc, partial, bytes;
    uint32_t nblocks;
};

inline uint64_t al256g(uint64_t x) { return (x + 255) & ~uint64_t(255); }

GsrLayout gsr_layout(int32_t n, int32_t m) {
    GsrLayout L;
    L.nblocks = ceil_div_u64(m > 0 ? (uint64_t)m : 1, kGsrThreads);
    uint64_t off = 0;
    L.rec = off; off = al256g(off + 16ull * kRec * n);
    L.acc = off; off = al256g(off + 4ull * kAcc * n);
    L.partial = off; off = al256g(off + 16ull * L.nblocks);
    L.bytes = off;
    return L;
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" size_t ges_gsr_workspace_bytes(int32_t n, int32_t m) {
    if (n < 1 || m < 1 || (uint64_t)n > (1ull << 26) || (uint64_t)m > (1ull << 28)) return 0;
    return gsr_layout(n, m).bytes;
}

extern "C" ges_status ges_gsr(int32_t n, const float *pos_op, const float *lscale_beta, const float *quat,
                              const ges_config *cfg, const int32_t *knn, int32_t m, const int32_t *sample_splat,
                              const float *sample_z, float lambda_sdf, float lambda_nor, void *workspace,
                              size_t workspace_bytes, float *losses, float *sample_out, float *g_pos_op,
                              float *g_lscale_beta, float *g_quat, void *stream) {
    GES_RANGE();
    if (n < 1 || m < 1 || (uint64_t)n > (1ull << 26) || (uint64_t)m > (1ull << 28)) return GES_ERR_INVALID_ARG;
    if (!pos_op || !lscale_beta || !quat || !cfg || !knn || !sample_splat || !sample_z || !workspace || !losses)
        return GES_ERR_INVALID_ARG;
    const bool grads = g_pos_op || g_lscale_beta || g_quat;
    if (grads && !(g_pos_op && g_lscale_beta && g_quat)) return GES_ERR_INVALID_ARG;
    for (const void *p : {(const void *)pos_op, (const void *)lscale_beta, (const void *)quat, (const void *)g_pos_op,
                          (const void *)g_lscale_beta, (const void *)g_quat})
        if ((uintptr_t)p & 15u) return GES_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 255u) || cfg->phi_mode < 0 || cfg->phi_mode > 2 || !isfinite(cfg->rho))
        return GES_ERR_INVALID_ARG;
    if (!isfinite(lambda_sdf) || !isfinite(lambda_nor)) return GES_ERR_INVALID_ARG;
    const GsrLayout L = gsr_layout(n, m);
    if (workspace_bytes < L.bytes) return GES_ERR_INVALID_ARG;
    GsrArgs a;
    memset(&a, 0, sizeof(a));
    a.n = n; a.m = m; a.phi_mode = cfg->phi_mode; a.rho = cfg->rho;
    a.pos_op = reinterpret_cast<const float4 *>(pos_op);
    a.lsb = reinterpret_cast<const float4 *>(lscale_beta);
    a.quat = reinterpret_cast<const float4 *>(quat);
    a.knn = knn; a.sample_splat = sample_splat; a.sample_z = sample_z;
    a.lambda_sdf = lambda_sdf; a.lambda_nor = lambda_nor; a.inv_m = (float)(1.0 / (double)m);
    char *ws = static_cast<char *>(workspace);
    a.rec = reinterpret_cast<float4 *>(ws + L.rec);
    a.acc = grads ? reinterpret_cast<float *>(ws + L.acc) : nullptr;
    a.partial = reinterpret_cast<double *>(ws + L.partial);
    a.losses = losses; a.sample_out = sample_out;
    a.g_pos_op = reinterpret_cast<float4 *>(g_pos_op);
    a.g_lsb = reinterpret_cast<float4 *>(g_lscale_beta);
    a.g_quat = reinterpret_cast<float4 *>(g_quat);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_gsr_prep<<<ceil_div_u64(n, 256), 256, 0, s>>>(a);
    k_gsr_sample<<<L.nblocks, kGsrThreads, 0, s>>>(a);
    k_gsr_finalize<<<1, 256, 0, s>>>(a, (int)L.nblocks);
    if (grads) k_gsr_chain<<<ceil_div_u64(n, 256), 256, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GES_OK : GES_ERR_CUDA;
}
