// Reconstruction loss of Eq. 8 (Sec. 3.2), L_rgb = (1 - lambda) L_1 + lambda L_SSIM,
// and its gradient with respect to the rendered colour, in one launch.
//
// One CTA per 32 x 32 output tile of a view, channels in turn. The SSIM gradient
// at a pixel q is a window sum over the pixels p around it of per-pixel
// derivatives of SSIM(p), which need the local statistics at p, which need the
// images around p: so the CTA stages both images on the tile plus two window
// radii (52 x 52) in shared memory, filters the five products x, y, x^2, y^2, xy
// with the separable 11-tap Gaussian (rows, then columns) to get the statistics on
// the tile plus one radius (42 x 42), forms SSIM and its three derivatives there,
// and filters those back onto the tile. Halo statistics are recomputed by the
// neighbouring CTAs rather than exchanged. Each CTA writes its partial sums of
// |x - y| and of SSIM to the workspace; a second launch adds them per view in a
// fixed order.
#include <cmath>
#include <cstring>

#include "ges_internal.cuh"

namespace ges {
namespace {

constexpr int kLT = 32;               // output tile side
constexpr int kR = 5;                 // window radius
constexpr int kWin = 2 * kR + 1;      // 11 taps
constexpr int kA = kLT + 4 * kR;      // 52: staged image region
constexpr int kB = kLT + 2 * kR;      // 42: statistics region
constexpr int kLossThreads = 384;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;
// row stride of the row-filtered products: 55 = 7 (mod 16) puts the 32 lanes of a column-pass read
// (consecutive columns, wrapping into the rows 6 below) on 32 distinct banks
constexpr int kBP = 55;
constexpr size_t kLossSmem = sizeof(float) * (2 * kA * kA + 5 * kA * kBP + 3 * kB * kB);
static_assert(kB % 6 == 0 && kLT % 4 == 0, "register blocking of the filter passes");

struct LossArgs {
    int n_views;
    int width[kMaxViews], height[kMaxViews], tiles_x[kMaxViews];
    int block_base[kMaxViews + 1];
    long long pix_base[kMaxViews + 1];
    float inv_n[kMaxViews];  // 1 / (3 W H)
    float gw[kWin];          // normalised 1-D window
    float lambda;
    const float *color, *target;
    float *g_color;
    double *partial;  // [blocks][2]
    float *loss;
};

__global__ void __launch_bounds__(kLossThreads) k_loss(const LossArgs a) {
    extern __shared__ float sm[];
    float *sx = sm;                // [kA][kA]
    float *sy = sx + kA * kA;      // [kA][kA]
    float *h1 = sy + kA * kA;       // [5][kA][kBP]: row-filtered products (kB used per row)
    float *st = h1 + 5 * kA * kBP;  // [3][kB][kB]: SSIM derivatives on the statistics region
    float *h2 = h1;                // [3][kB][kLT]: row-filtered derivatives (reuses h1)
    const int tid = threadIdx.x;
    const int b = blockIdx.x;
    int v = 0;
    while (v + 1 < a.n_views && b >= a.block_base[v + 1]) ++v;
    const int lb = b - a.block_base[v];
    const int W = a.width[v], H = a.height[v];
    const int tx0 = (lb % a.tiles_x[v]) * kLT, ty0 = (lb / a.tiles_x[v]) * kLT;
    const long long P = (long long)W * H;
    const float lam = a.lambda, inv_n = a.inv_n[v];
    float l1 = 0.f, ss = 0.f;  // this thread's few pixels; the CTA sum is formed in double
    for (int c = 0; c < 3; ++c) {
        const float *X = a.color + 3 * a.pix_base[v] + c * P;
        const float *Y = a.target + 3 * a.pix_base[v] + c * P;
        // images on the tile plus two radii; 0 outside the frame
        for (int i = tid; i < kA * kA; i += kLossThreads) {
            const int gy = ty0 - 2 * kR + i / kA, gx = tx0 - 2 * kR + i % kA;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            sx[i] = in ? __ldg(X + (long long)gy * W + gx) : 0.f;
            sy[i] = in ? __ldg(Y + (long long)gy * W + gx) : 0.f;
        }
        __syncthreads();
        // row pass of x, y, x^2, y^2, xy onto the statistics columns, 6 columns per
        // thread from a sliding window of 16 staged values
        for (int i = tid; i < kA * (kB / 6); i += kLossThreads) {
            const int ry = i / (kB / 6), c0 = (i % (kB / 6)) * 6;
            float xv[16], yv[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) { xv[k] = sx[ry * kA + c0 + k]; yv[k] = sy[ry * kA + c0 + k]; }
#pragma unroll
            for (int o = 0; o < 6; ++o) {
                float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
                for (int k = 0; k < kWin; ++k) {
                    const float w = a.gw[k];
                    const float wx = w * xv[o + k], wy = w * yv[o + k];
                    m0 += wx;
                    m1 += wy;
                    m2 = fmaf(wx, xv[o + k], m2);
                    m3 = fmaf(wy, yv[o + k], m3);
                    m4 = fmaf(wx, yv[o + k], m4);
                }
                const int j = ry * kBP + c0 + o;
                h1[j] = m0;
                h1[kA * kBP + j] = m1;
                h1[2 * kA * kBP + j] = m2;
                h1[3 * kA * kBP + j] = m3;
                h1[4 * kA * kBP + j] = m4;
            }
        }
        __syncthreads();
        // column pass, 6 rows per thread: local statistics, SSIM and its derivatives on
        // the statistics region
        for (int i = tid; i < kB * (kB / 6); i += kLossThreads) {
            const int cx = i % kB, r0 = (i / kB) * 6;
            float st5[5][6];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                float col[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) col[k] = h1[q * kA * kBP + (r0 + k) * kBP + cx];
#pragma unroll
                for (int o = 0; o < 6; ++o) {
                    float m = 0.f;
#pragma unroll
                    for (int k = 0; k < kWin; ++k) m = fmaf(a.gw[k], col[o + k], m);
                    st5[q][o] = m;
                }
            }
#pragma unroll
            for (int o = 0; o < 6; ++o) {
                const int r = r0 + o;
                const float mx = st5[0][o], my = st5[1][o];
                const int gy = ty0 - kR + r, gx = tx0 - kR + cx;
                const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
                const float sxx = st5[2][o] - mx * mx, syy = st5[3][o] - my * my, sxy = st5[4][o] - mx * my;
                const float n1 = 2.f * mx * my + kC1, n2 = 2.f * sxy + kC2;
                const float d1 = mx * mx + my * my + kC1, d2 = sxx + syy + kC2;
                const float id1 = __frcp_rn(d1), id2 = __frcp_rn(d2);
                const float s = n1 * n2 * id1 * id2;
                // dSSIM/dmu_x, dSSIM/ds_x^2, dSSIM/ds_xy; the first map below is the
                // coefficient of the window weight alone once s_x^2 and s_xy are expanded
                const float d_mx = 2.f * my * n2 * id1 * id2 - 2.f * mx * s * id1;
                const float d_sxx = -s * id2;
                const float d_sxy = 2.f * n1 * id1 * id2;
                const int j = r * kB + cx;
                st[j] = in ? d_mx - 2.f * d_sxx * mx - d_sxy * my : 0.f;
                st[kB * kB + j] = in ? d_sxx : 0.f;
                st[2 * kB * kB + j] = in ? d_sxy : 0.f;
                if (in && r >= kR && r < kR + kLT && cx >= kR && cx < kR + kLT) ss += s;
            }
        }
        __syncthreads();
        if (a.g_color) {
            // row pass of the derivatives onto the tile's columns, 4 per thread
            for (int i = tid; i < kB * (kLT / 4); i += kLossThreads) {
                const int r = i / (kLT / 4), c0 = (i % (kLT / 4)) * 4;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float row[14];
#pragma unroll
                    for (int k = 0; k < 14; ++k) row[k] = st[q * kB * kB + r * kB + c0 + k];
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        float f = 0.f;
#pragma unroll
                        for (int k = 0; k < kWin; ++k) f = fmaf(a.gw[k], row[o + k], f);
                        h2[q * kB * kLT + r * kLT + c0 + o] = f;
                    }
                }
            }
            __syncthreads();
            // column pass, 4 rows per thread, and the gradient
            float *G = a.g_color + 3 * a.pix_base[v] + c * P;
            for (int i = tid; i < kLT * (kLT / 4); i += kLossThreads) {
                const int ox = i % kLT, o0 = (i / kLT) * 4;
                float f[3][4];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float col[14];
#pragma unroll
                    for (int k = 0; k < 14; ++k) col[k] = h2[q * kB * kLT + (o0 + k) * kLT + ox];
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        float m = 0.f;
#pragma unroll
                        for (int k = 0; k < kWin; ++k) m = fmaf(a.gw[k], col[o + k], m);
                        f[q][o] = m;
                    }
                }
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int oy = o0 + o;
                    const int gy = ty0 + oy, gx = tx0 + ox;
                    if (gx >= W || gy >= H) continue;
                    const float xq = sx[(oy + 2 * kR) * kA + ox + 2 * kR], yq = sy[(oy + 2 * kR) * kA + ox + 2 * kR];
                    const float d = xq - yq;
                    const float sgn = (d > 0.f) ? 1.f : ((d < 0.f) ? -1.f : 0.f);
                    const float gs = f[0][o] + 2.f * xq * f[1][o] + yq * f[2][o];
                    G[(long long)gy * W + gx] = ((1.f - lam) * sgn - lam * gs) * inv_n;
                    l1 += fabsf(d);
                }
            }
        } else {
            for (int i = tid; i < kLT * (kLT / 4); i += kLossThreads) {
                const int ox = i % kLT, o0 = (i / kLT) * 4;
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int oy = o0 + o;
                    if (tx0 + ox >= W || ty0 + oy >= H) continue;
                    l1 += fabsf(sx[(oy + 2 * kR) * kA + ox + 2 * kR] - sy[(oy + 2 * kR) * kA + ox + 2 * kR]);
                }
            }
        }
        __syncthreads();  // the next channel overwrites the staged images
    }
    // CTA sums in a fixed order: warp shuffles, then warp 0 over the warps
    __shared__ double s_red[2][kLossThreads / 32];
    double dl1 = (double)l1, dss = (double)ss;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dl1 += __shfl_down_sync(0xffffffffu, dl1, o);
        dss += __shfl_down_sync(0xffffffffu, dss, o);
    }
    if ((tid & 31) == 0) { s_red[0][tid >> 5] = dl1; s_red[1][tid >> 5] = dss; }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int w = 0; w < kLossThreads / 32; ++w) { t0 += s_red[0][w]; t1 += s_red[1][w]; }
        a.partial[2 * (size_t)b] = t0;
        a.partial[2 * (size_t)b + 1] = t1;
    }
}

// Per view (one CTA each): the CTA partial sums, thread t taking blocks t, t + 256, ...,
// then a fixed tree over the threads; the order never depends on timing.
__global__ void __launch_bounds__(256) k_loss_finalize(const LossArgs a) {
    __shared__ double s0[256], s1[256];
    const int v = blockIdx.x, t = threadIdx.x;
    double l1 = 0.0, ss = 0.0;
    for (int b = a.block_base[v] + t; b < a.block_base[v + 1]; b += 256) {
        l1 += a.partial[2 * (size_t)b];
        ss += a.partial[2 * (size_t)b + 1];
    }
    s0[t] = l1;
    s1[t] = ss;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) { s0[t] += s0[t + o]; s1[t] += s1[t + o]; }
        __syncthreads();
    }
    if (t == 0) {
        const double n = 3.0 * (double)a.width[v] * (double)a.height[v];
        a.loss[v] = (float)((1.0 - (double)a.lambda) * s0[0] / n + (double)a.lambda * (1.0 - s1[0] / n));
    }
}

bool loss_views_ok(int32_t n_views, const ges_camera *cams) {
    if (n_views < 1 || n_views > kMaxViews || !cams) return false;
    for (int v = 0; v < n_views; ++v)
        if (cams[v].width < 1 || cams[v].height < 1 || cams[v].width > (1 << 15) || cams[v].height > (1 << 15))
            return false;
    return true;
}

int loss_blocks(int32_t n_views, const ges_camera *cams, LossArgs *a) {
    int nb = 0;
    long long pb = 0;
    for (int v = 0; v < n_views; ++v) {
        const int tx = (cams[v].width + kLT - 1) / kLT, ty = (cams[v].height + kLT - 1) / kLT;
        if (a) {
            a->width[v] = cams[v].width;
            a->height[v] = cams[v].height;
            a->tiles_x[v] = tx;
            a->block_base[v] = nb;
            a->pix_base[v] = pb;
            a->inv_n[v] = (float)(1.0 / (3.0 * (double)cams[v].width * (double)cams[v].height));
        }
        nb += tx * ty;
        pb += (long long)cams[v].width * cams[v].height;
    }
    if (a) {
        a->block_base[n_views] = nb;
        a->pix_base[n_views] = pb;
    }
    return nb;
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" size_t ges_loss_workspace_bytes(int32_t n_views, const ges_camera *cams) {
    if (!loss_views_ok(n_views, cams)) return 0;
    return sizeof(double) * 2 * (size_t)loss_blocks(n_views, cams, nullptr);
}

extern "C" ges_status ges_loss_rgb(int32_t n_views, const ges_camera *cams, const float *color, const float *target,
                                   float lambda, void *workspace, size_t workspace_bytes, float *loss, float *g_color,
                                   void *stream) {
    GES_RANGE();
    if (!loss_views_ok(n_views, cams) || !color || !target || !workspace || !loss) return GES_ERR_INVALID_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f)) return GES_ERR_INVALID_ARG;
    if (((uintptr_t)workspace & 7u) != 0) return GES_ERR_INVALID_ARG;
    LossArgs a;
    memset(&a, 0, sizeof(a));
    a.n_views = n_views;
    const int nb = loss_blocks(n_views, cams, &a);
    if (workspace_bytes < sizeof(double) * 2 * (size_t)nb) return GES_ERR_INVALID_ARG;
    double g[kWin], sum = 0.0;
    for (int k = 0; k < kWin; ++k) {
        const double d = (double)(k - kR);
        g[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[k];
    }
    for (int k = 0; k < kWin; ++k) a.gw[k] = (float)(g[k] / sum);
    a.lambda = lambda;
    a.color = color;
    a.target = target;
    a.g_color = g_color;
    a.partial = static_cast<double *>(workspace);
    a.loss = loss;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // 86 KB of dynamic shared memory (set on every call: the attribute belongs to the current device)
    if (cudaFuncSetAttribute(k_loss, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLossSmem) != cudaSuccess)
        return GES_ERR_CUDA;
    k_loss<<<nb, kLossThreads, kLossSmem, s>>>(a);
    k_loss_finalize<<<n_views, 256, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? GES_OK : GES_ERR_CUDA;
}
