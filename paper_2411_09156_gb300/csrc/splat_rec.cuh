// Per-splat frames and 80-byte records shared by the GSR evaluation and the level-set
// extraction: rotation of the normalised quaternion, phi-modulated scales, and a record
// (centre, opacity, rotation, 1/s'^2, beta, smallest scale and its axis) from which a
// point evaluates the splat's Mahalanobis form in the splat's own axes.
#pragma once

#include "ges_internal.cuh"

namespace ges {

constexpr int kRec = 5;  // float4 per splat record: (mu, o), R[0..3], R[4..7], (R[8], 1/s'^2), (beta, s_min, km, -)

// R (row-major, column k = axis k), s' = phi(beta) exp(l), dphi/dbeta, exp(l), 1/|q|, q/|q|.
__device__ __forceinline__ void splat_frame(const float4 *quat, const float4 *lsb, float rho, int phi_mode, int i,
                                            float *R, float *sp, float &dphi, float &phi, float *es, float &qinv,
                                            float *qn) {
    const float4 q4 = __ldg(quat + i), ls = __ldg(lsb + i);
    qinv = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    qn[0] = q4.x * qinv; qn[1] = q4.y * qinv; qn[2] = q4.z * qinv; qn[3] = q4.w * qinv;
    quat_rot(qn[0], qn[1], qn[2], qn[3], R);
    phi = phi_beta(ls.w, rho, phi_mode, dphi);
    es[0] = expf(ls.x); es[1] = expf(ls.y); es[2] = expf(ls.z);
    sp[0] = phi * es[0]; sp[1] = phi * es[1]; sp[2] = phi * es[2];
}

// Writes splat i's record.
__device__ __forceinline__ void build_splat_rec(const float4 *pos_op, const float4 *quat, const float4 *lsb, float rho,
                                                int phi_mode, int i, float4 *rec) {
    float R[9], sp[3], es[3], qn[4], dphi, phi, qinv;
    splat_frame(quat, lsb, rho, phi_mode, i, R, sp, dphi, phi, es, qinv, qn);
    const float4 po = __ldg(pos_op + i), ls = __ldg(lsb + i);
    int km = 0;
    if (ls.y < ls.x) km = 1;
    if (ls.z < (km == 0 ? ls.x : ls.y)) km = 2;
    const float smin = km == 0 ? sp[0] : (km == 1 ? sp[1] : sp[2]);
    float4 *r = rec + kRec * (size_t)i;
    r[0] = po;
    r[1] = make_float4(R[0], R[1], R[2], R[3]);
    r[2] = make_float4(R[4], R[5], R[6], R[7]);
    r[3] = make_float4(R[8], 1.f / (sp[0] * sp[0]), 1.f / (sp[1] * sp[1]), 1.f / (sp[2] * sp[2]));
    r[4] = make_float4(ls.w, smin, __int_as_float(km), 0.f);
}

// A splat record in registers.
struct NbRec {
    float4 r0;    // mu, o
    float R[9];   // rotation, row-major (column k = axis k)
    float ia[3];  // 1 / s'_k^2
    float beta, smin;
    int km;
};

__device__ __forceinline__ NbRec load_rec(const float4 *rec, int i) {
    const float4 *r = rec + kRec * (size_t)i;
    NbRec N;
    N.r0 = __ldg(r);
    const float4 a = __ldg(r + 1), b = __ldg(r + 2), c = __ldg(r + 3), d = __ldg(r + 4);
    N.R[0] = a.x; N.R[1] = a.y; N.R[2] = a.z; N.R[3] = a.w;
    N.R[4] = b.x; N.R[5] = b.y; N.R[6] = b.z; N.R[7] = b.w;
    N.R[8] = c.x; N.ia[0] = c.y; N.ia[1] = c.z; N.ia[2] = c.w;
    N.beta = d.x; N.smin = d.y; N.km = __float_as_int(d.z);
    return N;
}

}  // namespace ges
