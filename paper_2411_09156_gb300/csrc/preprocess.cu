// S1-S4 forward (projection, support, colour, normal, tile counts) and the
// S8 chain rule backward. One thread per splat; the splat's attributes are
// read once with float4 loads and every view is processed from registers, so a
// batch of V views reads the splat parameters once instead of V times.
#include "ges_internal.cuh"
#include "tile_tests.cuh"

namespace ges {


// ---------------------------------------------------------------------------
// S1: Sigma = R diag(s'^2) R^T with s' = phi(beta) exp(l)         (Eq. 4, 6-7)
// S2: t = W mu + t_w; J of the perspective map (clamped X/Z, Y/Z);
//     Sigma' = J W Sigma W^T J^T + h I; conic = Sigma'^-1          (Sec. 3.2)
// S3: q_cut = (2 ln(o / alpha_min))^(2/beta), the alpha_min level set of
//     exp(-1/2 Q^(beta/2))                                          (Eq. 3)
// S4: colour from SH, normal = R[:, argmin l] facing the camera   (Sec. 3.3)
//
// Sigma' is accumulated as sum_k s'_k^2 u_k u_k^T + h I with u_k = J W r_k the
// image of the splat's k-th axis: the same matrix as J W Sigma W^T J^T, without
// forming the 3x3 Sigma, whose tiny contribution along the flat axis of a
// flattened splat would be lost to float32 rounding.
//
// One thread per (splat, view), views innermost: the threads of one splat are
// adjacent, so its attributes are fetched from memory once per warp and the
// records of four splats x eight views are written as eight contiguous runs.
// ---------------------------------------------------------------------------
// Adds value f of a splat's flattened [16][3] coefficients (coefficient f / 3, channel f % 3).
__device__ __forceinline__ void sh_acc(int f, float x, const float *Y, float &r, float &g, float &b) {
    const int k = f / 3, ch = f % 3;
    if (ch == 0) r = fmaf(x, Y[k], r);
    else if (ch == 1) g = fmaf(x, Y[k], g);
    else b = fmaf(x, Y[k], b);
}

__device__ __forceinline__ void load_sh_rgb(const void *color, int st, int K, size_t i, const float *Y, float &r,
                                            float &g, float &b) {
    r = 0.5f; g = 0.5f; b = 0.5f;
    if (K == 16) {
        // each vector load is folded in at once (no 48-value array kept live)
        if (st == 0) {
            const float4 *c4 = reinterpret_cast<const float4 *>(static_cast<const float *>(color) + i * 48);
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                const float4 x = __ldg(c4 + q);
                sh_acc(4 * q, x.x, Y, r, g, b);
                sh_acc(4 * q + 1, x.y, Y, r, g, b);
                sh_acc(4 * q + 2, x.z, Y, r, g, b);
                sh_acc(4 * q + 3, x.w, Y, r, g, b);
            }
        } else {
            const uint4 *c16 = reinterpret_cast<const uint4 *>(static_cast<const char *>(color) + i * 96);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const uint4 u = __ldg(c16 + q);
                const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    sh_acc(8 * q + 2 * j, widen16(w[j] & 0xffffu, st), Y, r, g, b);
                    sh_acc(8 * q + 2 * j + 1, widen16(w[j] >> 16, st), Y, r, g, b);
                }
            }
        }
    } else {
        const size_t base = i * (size_t)K * 3;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (k < K) {
                r = fmaf(ld_color(color, st, base + 3 * k), Y[k], r);
                g = fmaf(ld_color(color, st, base + 3 * k + 1), Y[k], g);
                b = fmaf(ld_color(color, st, base + 3 * k + 2), Y[k], b);
            }
    }
    r = fmaxf(r, 0.f); g = fmaxf(g, 0.f); b = fmaxf(b, 0.f);
}

// Tile tests of a warp's 32 entries, spread over the warp's lanes (see
// warp_tile_rounds): each lane collects its own entry's hit count and, for the
// first 32 tests of its box, the row-major hit mask.
__device__ __forceinline__ void warp_tile_tests(const TileJob &J, int lane, int lw, int lh, int tw, int th,
                                                uint4 *jobs, uint32_t &tiles, uint32_t &mask) {
    tiles = 0;
    mask = 0;
    warp_tile_rounds(J, lane, lw, lh, tw, th, jobs,
                     [&](uint32_t hits, uint32_t lo, uint32_t len, uint32_t first, int, int, uint32_t, bool) {
                         if (!len) return;
                         const uint32_t bits = (hits >> lo) & (len == 32u ? 0xffffffffu : ((1u << len) - 1u));
                         tiles += (uint32_t)__popc(bits);
                         if (first < 32u) mask |= bits << first;  // bits of tests 32 and beyond drop out
                     });
}

// ST: the colour storage (Params::color_storage), a template parameter so that each storage
// gets its own register allocation.
template <int ST>
__global__ void __launch_bounds__(32, 32) k_preprocess(PreArgs a) {
    const uint32_t NV = (uint32_t)a.V.n_views;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;  // n * NV < 2^31 (host check)
    const int lane = threadIdx.x & 31;
    const bool live = t < (uint32_t)a.count * NV;
    const int tw = a.V.tile_w, th = a.V.tile_h;
    const int lw = __ffs(tw) - 1, lh = __ffs(th) - 1;  // tile sides are powers of two
    uint32_t i = 0, v = 0;
    size_t e = 0;
    float z32 = 0.f, ext_x = 0.f, ext_y = 0.f;
    bool visible = false;
    TileJob J = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, 0u};
    uint32_t rect = 0, rdim = 0;
    if (live) {
        const uint32_t il = t / NV;
        v = t - il * NV;
        i = (uint32_t)a.first + il;
        e = (size_t)v * a.n + i;
        if (v == 0 && a.P.sh_degree >= 0) {
            // the splat's colour coefficients (first and last byte: at most two lines for SH3) into
            // L2 while the projection runs, one lane per splat
            const int bytes = a.P.n_coeffs * 3 * (ST == 0 ? 4 : 2);
            const char *cb = static_cast<const char *>(a.color) + (size_t)i * bytes;
            prefetch_l2(cb);
            prefetch_l2(cb + bytes - 1);
        }
        const float4 po = __ldg(a.pos_op + i);
        const float4 ls = __ldg(a.lsb + i);
        const float4 q4 = __ldg(a.quat + i);
        const float o = po.w, beta = ls.w;
        const float *vm = a.V.vm[v];
        z32 = depth32(vm, po.x, po.y, po.z);
        float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
        // a splat with a non-finite position, opacity or shape, or beta <= 0, is culled and reported
        const bool in_ok = isfinite(po.x) && isfinite(po.y) && isfinite(po.z) && isfinite(o) && isfinite(beta) &&
                           beta > 0.f;
        if (!in_ok) set_error(a.err, kErrNumeric);
        const bool op_ok = o >= a.P.alpha_min;
        visible = in_ok && op_ok && z32 > a.V.znear[v];
        if (visible) {
            const float qinv = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
            float R[9];
            quat_rot(q4.x * qinv, q4.y * qinv, q4.z * qinv, q4.w * qinv, R);
            float dphi;
            const float phi = phi_beta(beta, a.P.rho, a.P.phi_mode, dphi);
            const float sx = phi * expf(ls.x), sy = phi * expf(ls.y), sz = phi * expf(ls.z);
            const float dk[3] = {sx * sx, sy * sy, sz * sz};
            const float qcut = powf(2.f * logf(o / a.P.alpha_min), 2.f / beta);
            const float qm = __fmul_rn(qcut, kSupportMargin);
            const float tx = vm[0] * po.x + vm[1] * po.y + vm[2] * po.z + vm[3];
            const float ty = vm[4] * po.x + vm[5] * po.y + vm[6] * po.z + vm[7];
            const float tz = z32;
            const float fx = a.V.fx[v], fy = a.V.fy[v];
            const float iz = 1.f / tz;
            const float rx = fminf(fmaxf(tx * iz, -a.V.limx[v]), a.V.limx[v]);
            const float ry = fminf(fmaxf(ty * iz, -a.V.limy[v]), a.V.limy[v]);
            const float J00 = fx * iz, J02 = -fx * rx * iz, J11 = fy * iz, J12 = -fy * ry * iz;
            const float T00 = J00 * vm[0] + J02 * vm[8], T01 = J00 * vm[1] + J02 * vm[9], T02 = J00 * vm[2] + J02 * vm[10];
            const float T10 = J11 * vm[4] + J12 * vm[8], T11 = J11 * vm[5] + J12 * vm[9], T12 = J11 * vm[6] + J12 * vm[10];
            // Sigma' = sum_k d_k u_k u_k^T + h I. Its determinant by the Cauchy-Binet sum
            // sum_{j<k} d_j d_k (u_j x u_k)^2 + h (A0 + C0) + h^2 has no cancellation, so the
            // conic of a long thin splat keeps float32 relative accuracy.
            float ux[3], uy[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ux[k] = T00 * R[k] + T01 * R[3 + k] + T02 * R[6 + k];
                uy[k] = T10 * R[k] + T11 * R[3 + k] + T12 * R[6 + k];
            }
            float A0 = 0.f, B = 0.f, C0 = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                A0 = fmaf(dk[k] * ux[k], ux[k], A0);
                B = fmaf(dk[k] * ux[k], uy[k], B);
                C0 = fmaf(dk[k] * uy[k], uy[k], C0);
            }
            const float x01 = ux[0] * uy[1] - uy[0] * ux[1];
            const float x02 = ux[0] * uy[2] - uy[0] * ux[2];
            const float x12 = ux[1] * uy[2] - uy[1] * ux[2];
            const float h = a.P.lowpass;
            const float A = A0 + h, C = C0 + h;
            const float det = dk[0] * dk[1] * x01 * x01 + dk[0] * dk[2] * x02 * x02 + dk[1] * dk[2] * x12 * x12 +
                              h * (A0 + C0) + h * h;
            const float idet = 1.f / det;
            const float ca = C * idet, cb = -B * idet, cc = A * idet;
            const float u = fx * tx * iz + a.V.cx[v];
            const float vv = fy * ty * iz + a.V.cy[v];
            if (!(det > 0.f) || !isfinite(ca) || !isfinite(cb) || !isfinite(cc) || !isfinite(u) || !isfinite(vv) ||
                !isfinite(qcut)) {
                visible = false;
                set_error(a.err, kErrNumeric);
            } else {
                ext_x = sqrtf(__fmul_rn(A, qm));
                ext_y = sqrtf(__fmul_rn(C, qm));
                // tile overlap (S3): the pixel box here, the ellipse-rectangle test per tile
                // of the box below (whole warp)
                int x0, x1, y0, y1;
                pixel_box(u, vv, ext_x, ext_y, a.V.width[v], a.V.height[v], x0, x1, y0, y1);
                if (x0 <= x1 && y0 <= y1) {
                    const int tx0 = x0 >> lw, tx1 = x1 >> lw, ty0 = y0 >> lh, ty1 = y1 >> lh;
                    const int rw = tx1 - tx0 + 1, rh = ty1 - ty0 + 1;
                    J = TileJob{u, vv, ca, cb, cc, __frcp_rn(ca), __frcp_rn(cc), qm,
                                (uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16),
                                (uint32_t)rw * (uint32_t)rh};
                    rect = (uint32_t)tx0 | ((uint32_t)ty0 << 16);
                    rdim = (uint32_t)rw | ((uint32_t)rh << 16);
                }
                // colour
                float rgb0, rgb1, rgb2;
                if (a.P.sh_degree >= 0) {
                    float dx = po.x - a.V.campos[v][0], dy = po.y - a.V.campos[v][1], dz = po.z - a.V.campos[v][2];
                    const float dinv = rsqrtf(dx * dx + dy * dy + dz * dz);
                    dx *= dinv; dy *= dinv; dz *= dinv;
                    float Y[16];
                    sh_eval(a.P.sh_degree, dx, dy, dz, Y);
                    load_sh_rgb(a.color, ST, a.P.n_coeffs, (size_t)i, Y, rgb0, rgb1, rgb2);
                } else {
                    rgb0 = ld_color(a.color, ST, 3 * (size_t)i);
                    rgb1 = ld_color(a.color, ST, 3 * (size_t)i + 1);
                    rgb2 = ld_color(a.color, ST, 3 * (size_t)i + 2);
                }
                // normal: axis of the smallest scale, facing the camera
                int ks = 0;
                if (ls.y < ls.x) ks = 1;
                if (ls.z < (ks == 0 ? ls.x : ls.y)) ks = 2;
                const float nx = ks == 0 ? R[0] : (ks == 1 ? R[1] : R[2]);
                const float ny = ks == 0 ? R[3] : (ks == 1 ? R[4] : R[5]);
                const float nz = ks == 0 ? R[6] : (ks == 1 ? R[7] : R[8]);
                const float f = nx * (a.V.campos[v][0] - po.x) + ny * (a.V.campos[v][1] - po.y) +
                                nz * (a.V.campos[v][2] - po.z);
                const float sg = f < 0.f ? -1.f : 1.f;
                r0 = make_float4(u, vv, ca, cb);
                r1 = make_float4(cc, qcut, 0.5f * beta, o);
                r2 = make_float4(rgb0, rgb1, rgb2, tz);
                r3 = make_float4(sg * nx, sg * ny, sg * nz, 0.f);
            }
        }
        a.rec[4 * e + 0] = r0;
        a.rec[4 * e + 1] = r1;
        a.rec[4 * e + 2] = r2;
        a.rec[4 * e + 3] = r3;
    }
    uint32_t tiles, mask;
    __shared__ uint4 s_jobs[1][kJobWords * 32];  // 32 threads: 1 warp
    warp_tile_tests(J, lane, lw, lh, tw, th, s_jobs[threadIdx.x >> 5], tiles, mask);
    unsigned long long my_tiles = 0;
    if (live) {
        const bool listed = visible && tiles > 0;
        const uint32_t key = listed ? __float_as_uint(z32) : kCulledKey;
        a.binrec[2 * e] = make_uint4(__float_as_uint(ext_x), __float_as_uint(ext_y), listed ? tiles : 0u, key);
        a.binrec[2 * e + 1] = make_uint4(mask, rect, rdim, 0u);
        my_tiles = listed ? tiles : 0u;
    }
    // tile count: a warp sum, one atomic per warp (a CTA is one warp)
    unsigned long long tsum = my_tiles;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tsum += __shfl_down_sync(0xffffffffu, tsum, off);
    if (lane == 0 && tsum) atomicAdd(a.total, tsum);
}

// ---------------------------------------------------------------------------
// S8: chain rule from the per-entry screen-space gradient g2d
// (u, v, a, b, c, o, beta, z, r, g, b, -, nx, ny, nz, -) to the 3-D inputs,
// summed over views in registers and written once (overwrite).
// ---------------------------------------------------------------------------

// Sum over the `width` lanes of a segment (width a power of two <= 32); every lane
// of the segment receives the sum.
__device__ __forceinline__ float seg_sum(float x, int width) {
    for (int o = width >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Recursive-halving sum of the 48 values wc_c Y_k (value 3k + c) over a segment of SEG lanes
// (compile-time sizes keep every index static, so the values stay in registers): at each level
// a lane keeps half of its values and adds its partner's copy of them, so 48 values cost
// 24 + 12 + ... shuffles instead of 48 per level. 48 = 3 x 16 halves four times; with 32 lanes
// the fifth level adds the 3 remaining values outright and the even lane of each pair writes.
// Lane v writes the sums it holds, values [base, base + CNT), that exist (index < 3K). At the
// first level value 3k + c pairs with 3(k + 8) + c, both wc_c times a basis value, so the lane
// takes Y_k and Y_k+8 in kept / sent order (16 selects) instead of swapping 24 product pairs.
template <int SEG>
__device__ __forceinline__ void write_sh_grad(const float (&wc)[3], const float (&Y)[16], int v, int K, bool ok,
                                              float *gcol) {
    constexpr int HALVINGS = SEG >= 16 ? 4 : (SEG == 8 ? 3 : (SEG == 4 ? 2 : (SEG == 2 ? 1 : 0)));
    constexpr int CNT = 48 >> HALVINGS;
    float t[48];
    int base = 0;
    if (HALVINGS == 0) {
#pragma unroll
        for (int k = 0; k < 16; ++k) { t[3 * k] = wc[0] * Y[k]; t[3 * k + 1] = wc[1] * Y[k]; t[3 * k + 2] = wc[2] * Y[k]; }
    } else {
        constexpr int o = SEG >> 1;
        const bool up = (v & o) != 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float yk = up ? Y[k + 8] : Y[k], ys = up ? Y[k] : Y[k + 8];
#pragma unroll
            for (int c = 0; c < 3; ++c) t[3 * k + c] = wc[c] * yk + __shfl_xor_sync(0xffffffffu, wc[c] * ys, o);
        }
        if (up) base += 24;
    }
#pragma unroll
    for (int l = 1, o = SEG >> 2, cnt = 24; l < HALVINGS; ++l, o >>= 1, cnt >>= 1) {
        const int h = cnt >> 1;
        const bool up = (v & o) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
            const float send = up ? t[q] : t[q + h];
            const float keep = up ? t[q + h] : t[q];
            t[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        if (up) base += h;
    }
    if (SEG == 32) {
#pragma unroll
        for (int q = 0; q < CNT; ++q) t[q] += __shfl_xor_sync(0xffffffffu, t[q], 1);
    }
    if (ok && (SEG < 32 || (v & 1) == 0)) {
#pragma unroll
        for (int q = 0; q < CNT; ++q)
            if (base + q < K * 3) gcol[base + q] = t[q];
    }
}

// Per-splat stride (floats) of the staged SH coefficients: the 3K floats rounded up to whole
// float4s, an odd number of them, so that the staged splats of a warp start in distinct bank
// groups (a stride of 48 floats put every other splat on the same banks).
__host__ __device__ __forceinline__ int sh_stage_stride(int K) {
    int s4 = (K * 3 + 3) / 4;
    if ((s4 & 1) == 0) ++s4;
    return 4 * s4;
}

// One lane per (splat, view): the lanes of a splat are adjacent (a segment of
// `seg` lanes, the view count rounded up to a power of two), each lane takes its
// view's screen-space gradient back through S1-S4, and the per-splat sums over
// views are formed with shuffles inside the segment. Lane 0 of the segment
// writes the geometry gradients; the SH coefficient gradients are written by all
// lanes of the segment, coefficient k by lane k mod seg.
template <int SEG>
__global__ void __launch_bounds__(32, 28) k_preprocess_bwd(PreBwdArgs a) {
    const int NV = a.V.n_views;
    constexpr int seg = SEG;  // lanes per splat: the view count rounded up to a power of two
    const int lane = threadIdx.x & 31;
    const int spw = 32 / seg;  // splats per warp
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int v = lane % seg;
    const long long end = (long long)a.first + a.count;
    const long long il = a.first + gw * spw + lane / seg;
    if (gw * spw >= a.count) return;  // whole warp past the end (warp-uniform)
    const bool splat_ok = il < end;
    const int i = splat_ok ? (int)il : (int)(end - 1);
    const bool active = splat_ok && v < NV;
    // the SH coefficients of the warp's splats, loaded once with coalesced float4 reads
    // (dynamic shared memory: spw * K * 3 floats per warp)
    extern __shared__ float s_sh[];
    const int K = a.P.n_coeffs;
    const int S = sh_stage_stride(K), K3 = K * 3;
    float *wsh = s_sh + (threadIdx.x >> 5) * (spw * S);
    if (a.P.sh_degree >= 0) {
        const long long first = a.first + gw * spw;
        const int nsp = (int)min((long long)spw, end - first);
        const int nflt = nsp * K * 3;
        const int st = a.P.color_storage;
        const size_t off = (size_t)first * K * 3;
        // flat float f of the run goes to splat f / 3K, offset f % 3K (a float4 or a 16-byte chunk
        // of 16-bit values never straddles two splats on those paths)
        if (st == 0 && K3 % 4 == 0) {
            const float4 *s4 = reinterpret_cast<const float4 *>(static_cast<const float *>(a.color) + off);
            for (int q = lane; q < nflt / 4; q += 32) {
                const int sp = 4 * q / K3;
                *reinterpret_cast<float4 *>(wsh + sp * S + (4 * q - sp * K3)) = __ldg(s4 + q);
            }
        } else if (st != 0 && K3 % 8 == 0) {
            const char *s16 = static_cast<const char *>(a.color) + 2 * off;
            for (int q = lane; q < nflt / 8; q += 32) {
                const int sp = 8 * q / K3;
                ld_color8(s16 + 16 * q, st, wsh + sp * S + (8 * q - sp * K3));
            }
        } else {
            for (int q = lane; q < nflt; q += 32) {
                const int sp = q / K3;
                wsh[sp * S + (q - sp * K3)] = ld_color(a.color, st, off + q);
            }
        }
        __syncwarp();
    }
    const float *cf = wsh + (lane / seg) * S;  // this lane's splat
    const float4 po = __ldg(a.pos_op + i);
    const float4 ls = __ldg(a.lsb + i);
    const float4 q4 = __ldg(a.quat + i);
    const float beta = ls.w;
    const float qinv = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float qw = q4.x * qinv, qx = q4.y * qinv, qy = q4.z * qinv, qz = q4.w * qinv;
    float R[9];
    quat_rot(qw, qx, qy, qz, R);
    float dphi;
    const float phi = phi_beta(beta, a.P.rho, a.P.phi_mode, dphi);
    const float e0 = expf(ls.x), e1 = expf(ls.y), e2 = expf(ls.z);
    const float sp[3] = {phi * e0, phi * e1, phi * e2};
    const float es[3] = {e0, e1, e2};
    const float dd[3] = {sp[0] * sp[0], sp[1] * sp[1], sp[2] * sp[2]};
    int ks = 0;
    if (ls.y < ls.x) ks = 1;
    if (ls.z < (ks == 0 ? ls.x : ls.y)) ks = 2;
    // this lane's view
    float gmu[3] = {0.f, 0.f, 0.f}, gop = 0.f, gbeta = 0.f;
    float GR[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float gD[3] = {0.f, 0.f, 0.f};  // dL/d(s'_k^2)
    float wc[3] = {0.f, 0.f, 0.f};  // colour gradient where the channel was not clamped
    float sdir[3] = {0.f, 0.f, 0.f};
    bool has = false;
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0, g2 = g0, g3 = g0;
    if (active) {
        const size_t e = (size_t)v * a.n + i;
        g0 = a.g2d[4 * e + 0]; g1 = a.g2d[4 * e + 1]; g2 = a.g2d[4 * e + 2]; g3 = a.g2d[4 * e + 3];
        has = !(g0.x == 0.f && g0.y == 0.f && g0.z == 0.f && g0.w == 0.f && g1.x == 0.f && g1.y == 0.f &&
                g1.z == 0.f && g1.w == 0.f && g2.x == 0.f && g2.y == 0.f && g2.z == 0.f && g3.x == 0.f &&
                g3.y == 0.f && g3.z == 0.f);
    }
    if (has) {
        const float *vm = a.V.vm[v];
        const float tx = vm[0] * po.x + vm[1] * po.y + vm[2] * po.z + vm[3];
        const float ty = vm[4] * po.x + vm[5] * po.y + vm[6] * po.z + vm[7];
        const float tz = depth32(vm, po.x, po.y, po.z);
        const float fx = a.V.fx[v], fy = a.V.fy[v];
        const float iz = 1.f / tz;
        const float rxr = tx * iz, ryr = ty * iz;
        const bool clx = rxr < -a.V.limx[v] || rxr > a.V.limx[v];
        const bool cly = ryr < -a.V.limy[v] || ryr > a.V.limy[v];
        const float rx = fminf(fmaxf(rxr, -a.V.limx[v]), a.V.limx[v]);
        const float ry = fminf(fmaxf(ryr, -a.V.limy[v]), a.V.limy[v]);
        const float J00 = fx * iz, J02 = -fx * rx * iz, J11 = fy * iz, J12 = -fy * ry * iz;
        const float T[6] = {J00 * vm[0] + J02 * vm[8], J00 * vm[1] + J02 * vm[9], J00 * vm[2] + J02 * vm[10],
                            J11 * vm[4] + J12 * vm[8], J11 * vm[5] + J12 * vm[9], J11 * vm[6] + J12 * vm[10]};
        // dL/dSigma' (symmetric-matrix gradient) as accumulated by the render backward
        const float M00 = g0.z, M01 = g0.w, M11 = g1.x;
        // Sigma' = sum_k s'_k^2 u_k u_k^T + h I with u_k = T r_k. With w_k = G_M u_k:
        //   dL/d(s'_k^2) += u_k . w_k,  dL/dR[:, k] += 2 s'_k^2 T^T w_k,
        //   dL/dT = 2 sum_k s'_k^2 w_k r_k^T
        float GT[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float ux = T[0] * R[k] + T[1] * R[3 + k] + T[2] * R[6 + k];
            const float uy = T[3] * R[k] + T[4] * R[3 + k] + T[5] * R[6 + k];
            const float wx = M00 * ux + M01 * uy, wy = M01 * ux + M11 * uy;
            gD[k] = ux * wx + uy * wy;
            const float s2 = 2.f * dd[k];
            GR[0 + k] = s2 * (T[0] * wx + T[3] * wy);
            GR[3 + k] = s2 * (T[1] * wx + T[4] * wy);
            GR[6 + k] = s2 * (T[2] * wx + T[5] * wy);
            GT[0] += s2 * wx * R[k]; GT[1] += s2 * wx * R[3 + k]; GT[2] += s2 * wx * R[6 + k];
            GT[3] += s2 * wy * R[k]; GT[4] += s2 * wy * R[3 + k]; GT[5] += s2 * wy * R[6 + k];
        }
        // T = J W: G_J = G_T W^T (only the non-zero entries of J matter)
        const float GJ00 = GT[0] * vm[0] + GT[1] * vm[1] + GT[2] * vm[2];
        const float GJ02 = GT[0] * vm[8] + GT[1] * vm[9] + GT[2] * vm[10];
        const float GJ11 = GT[3] * vm[4] + GT[4] * vm[5] + GT[5] * vm[6];
        const float GJ12 = GT[3] * vm[8] + GT[4] * vm[9] + GT[5] * vm[10];
        const float iz2 = iz * iz, iz3 = iz2 * iz;
        float gt0 = 0.f, gt1 = 0.f, gt2 = 0.f;
        gt2 += -fx * iz2 * GJ00 - fy * iz2 * GJ11;
        if (!clx) { gt0 += -fx * iz2 * GJ02; gt2 += 2.f * fx * tx * iz3 * GJ02; }
        else gt2 += fx * rx * iz2 * GJ02;
        if (!cly) { gt1 += -fy * iz2 * GJ12; gt2 += 2.f * fy * ty * iz3 * GJ12; }
        else gt2 += fy * ry * iz2 * GJ12;
        // mean and depth value
        gt0 += fx * iz * g0.x; gt2 += -fx * tx * iz2 * g0.x;
        gt1 += fy * iz * g0.y; gt2 += -fy * ty * iz2 * g0.y;
        gt2 += g1.w;
        gmu[0] = vm[0] * gt0 + vm[4] * gt1 + vm[8] * gt2;
        gmu[1] = vm[1] * gt0 + vm[5] * gt1 + vm[9] * gt2;
        gmu[2] = vm[2] * gt0 + vm[6] * gt1 + vm[10] * gt2;
        gop = g1.y;
        gbeta = g1.z;
        // normal: n = sign R[:, ks] (column chosen with selects: a runtime index would
        // move R and GR to local memory)
        const float nx = ks == 0 ? R[0] : (ks == 1 ? R[1] : R[2]);
        const float ny = ks == 0 ? R[3] : (ks == 1 ? R[4] : R[5]);
        const float nz = ks == 0 ? R[6] : (ks == 1 ? R[7] : R[8]);
        const float f = nx * (a.V.campos[v][0] - po.x) + ny * (a.V.campos[v][1] - po.y) + nz * (a.V.campos[v][2] - po.z);
        const float sg = f < 0.f ? -1.f : 1.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float on = (ks == c) ? sg : 0.f;
            GR[0 + c] += on * g3.x;
            GR[3 + c] += on * g3.y;
            GR[6 + c] += on * g3.z;
        }
        // colour
        if (a.P.sh_degree >= 0) {
            float dx = po.x - a.V.campos[v][0], dy = po.y - a.V.campos[v][1], dz = po.z - a.V.campos[v][2];
            const float dinv = rsqrtf(dx * dx + dy * dy + dz * dz);
            dx *= dinv; dy *= dinv; dz *= dinv;
            sdir[0] = dx; sdir[1] = dy; sdir[2] = dz;
            float Y[16];
            sh_eval(a.P.sh_degree, dx, dy, dz, Y);
            const float gc[3] = {g2.x, g2.y, g2.z};
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float pre = 0.5f;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < K) pre = fmaf(cf[3 * k + ch], Y[k], pre);
                if (pre > 0.f) wc[ch] = gc[ch];
            }
            // d/dd of sum_c wc_c sum_k c_kc Y_k(d): one polynomial with coefficients al_k
            float al[16];
#pragma unroll
            for (int k = 0; k < 16; ++k)
                al[k] = (k < K) ? wc[0] * cf[3 * k] + wc[1] * cf[3 * k + 1] + wc[2] * cf[3 * k + 2] : 0.f;
            float gd0, gd1, gd2;
            sh_grad_dot(a.P.sh_degree, dx, dy, dz, al, gd0, gd1, gd2);
            const float dot = gd0 * dx + gd1 * dy + gd2 * dz;
            gmu[0] += (gd0 - dx * dot) * dinv;
            gmu[1] += (gd1 - dy * dot) * dinv;
            gmu[2] += (gd2 - dz * dot) * dinv;
        } else {
            wc[0] = g2.x; wc[1] = g2.y; wc[2] = g2.z;
        }
    }
    // sums over the views of this splat
#pragma unroll
    for (int k = 0; k < 3; ++k) { gmu[k] = seg_sum(gmu[k], seg); gD[k] = seg_sum(gD[k], seg); }
#pragma unroll
    for (int k = 0; k < 9; ++k) GR[k] = seg_sum(GR[k], seg);
    gop = seg_sum(gop, seg);
    gbeta = seg_sum(gbeta, seg);
    // a splat with no screen-space gradient in any view (culled, or reaching no pixel with an
    // upstream gradient) has zero 3-D gradients, whatever its parameters (a culled splat may hold
    // non-finite ones)
    const bool any_view = seg_sum(has ? 1.f : 0.f, seg) > 0.f;
    if (splat_ok && v == 0 && !any_view) {
        a.g_quat[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        a.g_pos_op[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        a.g_lsb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else if (splat_ok && v == 0) {
        // s'_k = phi(beta) exp(l_k): dL/dl_k = 2 s'_k^2 gD_k, dL/dbeta += 2 s'_k gD_k phi'(beta) exp(l_k)
        float gl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float gsp = 2.f * sp[k] * gD[k];
            gl[k] = gsp * sp[k];
            gbeta += gsp * dphi * es[k];
        }
        // R(q) -> unit quaternion -> quaternion
        const float w = qw, x = qx, y = qy, z = qz;
        const float gw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
        const float gx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] - 2.f * x * GR[8]);
        const float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] - 2.f * y * GR[8]);
        const float gz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] + x * GR[6] + y * GR[7]);
        const float dq = gw * w + gx * x + gy * y + gz * z;
        a.g_quat[i] = make_float4((gw - w * dq) * qinv, (gx - x * dq) * qinv, (gy - y * dq) * qinv, (gz - z * dq) * qinv);
        a.g_pos_op[i] = make_float4(gmu[0], gmu[1], gmu[2], gop);
        a.g_lsb[i] = make_float4(gl[0], gl[1], gl[2], gbeta);
    }
    // colour coefficients: dL/dc_kc = sum_v wc_vc Y_k(d_v) (RGB mode: sum_v wc_vc)
    if (a.P.sh_degree < 0) {
        float s0 = seg_sum(wc[0], seg), s1 = seg_sum(wc[1], seg), s2 = seg_sum(wc[2], seg);
        if (splat_ok && v == 0) { a.g_color[3 * (size_t)i] = s0; a.g_color[3 * (size_t)i + 1] = s1; a.g_color[3 * (size_t)i + 2] = s2; }
        return;
    }
    float Y[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) Y[k] = 0.f;
    if (has) sh_eval(a.P.sh_degree, sdir[0], sdir[1], sdir[2], Y);
    // the 48 products wc_c Y_k summed over the segment's lanes
    write_sh_grad<SEG>(wc, Y, v, K, splat_ok, a.g_color + (size_t)i * K * 3);
}

cudaError_t launch_preprocess(const PreArgs &a, cudaStream_t s) {
    if (a.count <= 0) return cudaSuccess;
    const long long threads = (long long)a.count * a.V.n_views;
    // one warp per CTA: the warps share nothing but the SM, so a warp whose tile tests end early
    // frees its slot at once (0.93 -> 0.83 ms against CTAs of 8 warps)
    const unsigned grid = (unsigned)((threads + 31) / 32);
    if (a.P.color_storage == 1) k_preprocess<1><<<grid, 32, 0, s>>>(a);
    else if (a.P.color_storage == 2) k_preprocess<2><<<grid, 32, 0, s>>>(a);
    else k_preprocess<0><<<grid, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const PreBwdArgs &a, cudaStream_t s) {
    if (a.count <= 0) return cudaSuccess;
    int seg = 1;
    while (seg < a.V.n_views) seg <<= 1;
    const long long warps = ((long long)a.count + (32 / seg) - 1) / (32 / seg);
    // one warp per CTA, 28 resident per SM (72 registers: more resident warps hide the
    // loads better than the few spills cost; 0.85 -> 0.75 ms against CTAs of 8 warps)
    const size_t smem = a.P.sh_degree >= 0 ? (size_t)(32 / seg) * sh_stage_stride(a.P.n_coeffs) * sizeof(float) : 0;
    const unsigned grid = (unsigned)warps;
    switch (seg) {
        case 1: k_preprocess_bwd<1><<<grid, 32, smem, s>>>(a); break;
        case 2: k_preprocess_bwd<2><<<grid, 32, smem, s>>>(a); break;
        case 4: k_preprocess_bwd<4><<<grid, 32, smem, s>>>(a); break;
        case 8: k_preprocess_bwd<8><<<grid, 32, smem, s>>>(a); break;
        case 16: k_preprocess_bwd<16><<<grid, 32, smem, s>>>(a); break;
        default: k_preprocess_bwd<32><<<grid, 32, smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace ges
