// C ABI of libges.so (declared and documented in include/ges.h): host-side
// argument checks, buffer layouts and kernel launches on the caller's stream.
// The library owns no memory; every buffer is passed in by the caller.
#include <math.h>
#include <string.h>

#include "ges_internal.cuh"

using namespace ges;

namespace {

constexpr uint64_t kMaxEntries = (uint64_t)kScanTile * kScanMaxPartials;  // 67,108,864 (view, splat) entries

bool finite_pos(float x) { return isfinite(x) && x > 0.f; }

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bool check_config(const ges_config *cfg) {
    if (!cfg) return false;
    if (!tile_shape_supported(cfg->tile_w, cfg->tile_h)) return false;
    if (cfg->batch < 32 || cfg->batch > 256 || (cfg->batch & 31)) return false;
    if (cfg->sh_degree < -1 || cfg->sh_degree > 3) return false;
    if (cfg->phi_mode < 0 || cfg->phi_mode > 2) return false;
    if (!isfinite(cfg->rho) || !isfinite(cfg->lowpass) || cfg->lowpass < 0.f) return false;
    if (!(cfg->alpha_min > 0.f && cfg->alpha_min < 1.f)) return false;
    if (!(cfg->alpha_max >= cfg->alpha_min && cfg->alpha_max < 1.f)) return false;
    if (!(cfg->t_min >= 0.f && cfg->t_min < 1.f)) return false;
    if (!finite_pos(cfg->jac_clamp)) return false;
    for (int c = 0; c < 3; ++c)
        if (!isfinite(cfg->bg[c])) return false;
    if (cfg->persistent != 0 && cfg->persistent != 1) return false;
    if (cfg->color_storage < 0 || cfg->color_storage > 2) return false;
    return true;
}

bool check_views(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg) {
    if (n < 0 || n_views < 1 || n_views > kMaxViews || !cams || !check_config(cfg)) return false;
    if ((uint64_t)n * (uint64_t)n_views > kMaxEntries) return false;
    uint64_t tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const ges_camera &c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > (1 << 15) || c.height > (1 << 15)) return false;
        if (!finite_pos(c.fx) || !finite_pos(c.fy) || !isfinite(c.cx) || !isfinite(c.cy)) return false;
        if (!finite_pos(c.znear)) return false;
        for (int k = 0; k < 12; ++k)
            if (!isfinite(c.viewmat[k])) return false;
        tiles += (uint64_t)((c.width + cfg->tile_w - 1) / cfg->tile_w) * ((c.height + cfg->tile_h - 1) / cfg->tile_h);
        pix += (uint64_t)c.width * c.height;
    }
    return tiles < (1ull << 31) && pix < (1ull << 40);
}

ViewSet make_views(int32_t n_views, const ges_camera *cams, const ges_config *cfg) {
    ViewSet V;
    memset(&V, 0, sizeof(V));
    V.n_views = n_views;
    V.tile_w = cfg->tile_w;
    V.tile_h = cfg->tile_h;
    int tb = 0;
    long long pb = 0;
    for (int v = 0; v < n_views; ++v) {
        const ges_camera &c = cams[v];
        V.width[v] = c.width;
        V.height[v] = c.height;
        V.tiles_x[v] = (c.width + cfg->tile_w - 1) / cfg->tile_w;
        const int tiles_y = (c.height + cfg->tile_h - 1) / cfg->tile_h;
        V.tile_base[v] = tb;
        V.pix_base[v] = pb;
        tb += V.tiles_x[v] * tiles_y;
        pb += (long long)c.width * c.height;
        V.fx[v] = c.fx; V.fy[v] = c.fy; V.cx[v] = c.cx; V.cy[v] = c.cy;
        for (int k = 0; k < 12; ++k) V.vm[v][k] = c.viewmat[k];
        V.znear[v] = c.znear;
        V.limx[v] = cfg->jac_clamp * 0.5f * (float)c.width / c.fx;
        V.limy[v] = cfg->jac_clamp * 0.5f * (float)c.height / c.fy;
        for (int j = 0; j < 3; ++j)  // camera centre -R^T t
            V.campos[v][j] = -(c.viewmat[0 * 4 + j] * c.viewmat[3] + c.viewmat[1 * 4 + j] * c.viewmat[7] +
                               c.viewmat[2 * 4 + j] * c.viewmat[11]);
    }
    V.tile_base[n_views] = tb;
    V.pix_base[n_views] = pb;
    V.n_tiles = tb;
    return V;
}

Params make_params(const ges_config *cfg) {
    Params P;
    P.sh_degree = cfg->sh_degree;
    P.n_coeffs = cfg->sh_degree < 0 ? 1 : (cfg->sh_degree + 1) * (cfg->sh_degree + 1);
    P.phi_mode = cfg->phi_mode;
    P.rho = cfg->rho;
    P.lowpass = cfg->lowpass;
    P.alpha_min = cfg->alpha_min;
    P.alpha_max = cfg->alpha_max;
    P.t_min = cfg->t_min;
    for (int c = 0; c < 3; ++c) P.bg[c] = cfg->bg[c];
    P.color_storage = cfg->color_storage;
    return P;
}

// Largest instance capacity whose layout fits in `bytes`.
uint64_t capacity_for(int32_t n, int32_t n_views, uint32_t n_tiles, size_t bytes) {
    if (bins_layout(n, n_views, n_tiles, 0).bytes > bytes) return UINT64_MAX;  // does not fit at all
    uint64_t lo = 0, hi = 0xfffffffeull;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo + 1) / 2;
        if (bins_layout(n, n_views, n_tiles, mid).bytes <= bytes) lo = mid; else hi = mid - 1;
    }
    return lo;
}

ges_status cuda_status(cudaError_t e) { return e == cudaSuccess ? GES_OK : GES_ERR_CUDA; }

template <typename T>
T *at(void *base, uint64_t off) { return reinterpret_cast<T *>(static_cast<char *>(base) + off); }
template <typename T>
const T *at(const void *base, uint64_t off) { return reinterpret_cast<const T *>(static_cast<const char *>(base) + off); }

}  // namespace

extern "C" {

int32_t ges_abi_version(void) { return GES_ABI_VERSION; }

int32_t ges_build_flags(void) {
#ifdef GES_DEBUG
    return GES_BUILD_DEBUG;
#else
    return 0;
#endif
}

const char *ges_status_string(ges_status s) {
    switch (s) {
        case GES_OK: return "ok";
        case GES_ERR_INVALID_ARG: return "invalid argument";
        case GES_ERR_CAPACITY: return "tile-instance capacity exceeded; lists truncated";
        case GES_ERR_CUDA: return "CUDA error";
        case GES_ERR_NUMERIC: return "non-finite input or projection; splat culled";
        case GES_ERR_TOO_LARGE: return "problem exceeds the fixed scratch of the no-allocation entry point";
        case GES_ERR_BOUNDS: return "device-side bounds check failed (debug build); access skipped";
        default: return "unknown status";
    }
}

size_t ges_proj_bytes(int32_t n, int32_t n_views) {
    if (n < 0 || n_views < 1 || n_views > kMaxViews || (uint64_t)n * n_views > kMaxEntries) return 0;
    return (size_t)proj_layout(n, n_views).bytes;
}

size_t ges_bins_bytes(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg, uint64_t capacity) {
    if (!check_views(n, n_views, cams, cfg) || capacity > 0xfffffffeull) return 0;
    const ViewSet V = make_views(n_views, cams, cfg);
    const BinsLayout L = bins_layout(n, n_views, (uint32_t)V.n_tiles, capacity);
    if ((uint64_t)256 * L.nblk_inst > kMaxEntries) return 0;
    return (size_t)L.bytes;
}

ges_status ges_get_layout(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                          uint64_t capacity, ges_layout *out) {
    GES_RANGE();
    if (!out || !check_views(n, n_views, cams, cfg) || capacity > 0xfffffffeull) return GES_ERR_INVALID_ARG;
    const ViewSet V = make_views(n_views, cams, cfg);
    const ProjLayout P = proj_layout(n, n_views);
    const BinsLayout B = bins_layout(n, n_views, (uint32_t)V.n_tiles, capacity);
    memset(out, 0, sizeof(*out));
    out->proj_records = P.records;
    out->proj_binrec = P.binrec;
    out->proj_g2d = P.g2d;
    out->proj_bytes = P.bytes;
    const int res = B.tile_passes & 1;
    out->bins_inst_tile = B.ikey[res];
    out->bins_inst_entry = B.ival[res];
    out->bins_ranges = B.ranges;
    out->bins_queue = B.queue;
    out->bins_bytes = B.bytes;
    out->n_tiles = (uint32_t)V.n_tiles;
    for (int v = 0; v < n_views; ++v) out->tile_base[v] = (uint32_t)V.tile_base[v];
    return GES_OK;
}

// S1-S4 for the splats [first, first + count) of n; the range starting at 0 clears the header.
static ges_status preprocess_impl(int32_t n, int32_t first, int32_t count, const float *pos_op,
                                  const float *lscale_beta, const float *quat, const void *color, int32_t n_views,
                                  const ges_camera *cams, const ges_config *cfg, void *proj, size_t proj_bytes,
                                  void *stream) {
    if (!check_views(n, n_views, cams, cfg) || !proj || !aligned16(proj)) return GES_ERR_INVALID_ARG;
    if (first < 0 || count < 0 || (int64_t)first + count > n) return GES_ERR_INVALID_ARG;
    const ProjLayout L = proj_layout(n, n_views);
    if (proj_bytes < L.bytes) return GES_ERR_INVALID_ARG;
    if (n > 0 && (!pos_op || !lscale_beta || !quat || !color || !aligned16(pos_op) || !aligned16(lscale_beta) ||
                  !aligned16(quat) || !aligned16(color)))
        return GES_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (first == 0 && cudaMemsetAsync(proj, 0, 16, s) != cudaSuccess) return GES_ERR_CUDA;  // total + error word
    PreArgs a;
    a.n = n;
    a.first = first;
    a.count = count;
    a.pos_op = reinterpret_cast<const float4 *>(pos_op);
    a.lsb = reinterpret_cast<const float4 *>(lscale_beta);
    a.quat = reinterpret_cast<const float4 *>(quat);
    a.color = color;
    a.rec = at<float4>(proj, L.records);
    a.binrec = at<uint4>(proj, L.binrec);
    a.total = at<unsigned long long>(proj, 0);
    a.err = at<uint32_t>(proj, 8);
    a.P = make_params(cfg);
    a.V = make_views(n_views, cams, cfg);
    return cuda_status(launch_preprocess(a, s));
}

ges_status ges_preprocess(int32_t n, const float *pos_op, const float *lscale_beta, const float *quat,
                          const void *color, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                          void *proj, size_t proj_bytes, void *stream) {
    GES_RANGE();
    return preprocess_impl(n, 0, n, pos_op, lscale_beta, quat, color, n_views, cams, cfg, proj, proj_bytes, stream);
}

ges_status ges_preprocess_range(int32_t n, int32_t first, int32_t count, const float *pos_op,
                                const float *lscale_beta, const float *quat, const void *color, int32_t n_views,
                                const ges_camera *cams, const ges_config *cfg, void *proj, size_t proj_bytes,
                                void *stream) {
    GES_RANGE();
    return preprocess_impl(n, first, count, pos_op, lscale_beta, quat, color, n_views, cams, cfg, proj, proj_bytes,
                           stream);
}

ges_status ges_instance_count(const void *proj, size_t proj_bytes, uint64_t *count, void *stream) {
    GES_RANGE();
    if (!proj || !count || proj_bytes < 256) return GES_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long v = 0;
    if (cudaMemcpyAsync(&v, proj, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess) return GES_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GES_ERR_CUDA;
    *count = v;
    return GES_OK;
}

ges_status ges_bin(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg, void *proj,
                   size_t proj_bytes, void *bins, size_t bins_bytes, void *stream) {
    GES_RANGE();
    if (!check_views(n, n_views, cams, cfg) || !proj || !bins || !aligned16(proj) || !aligned16(bins))
        return GES_ERR_INVALID_ARG;
    const ProjLayout PL = proj_layout(n, n_views);
    if (proj_bytes < PL.bytes) return GES_ERR_INVALID_ARG;
    const ViewSet V = make_views(n_views, cams, cfg);
    const uint64_t cap = capacity_for(n, n_views, (uint32_t)V.n_tiles, bins_bytes);
    if (cap == UINT64_MAX) return GES_ERR_INVALID_ARG;
    const BinsLayout L = bins_layout(n, n_views, (uint32_t)V.n_tiles, cap);
    if ((uint64_t)256 * L.nblk_inst > kMaxEntries) return GES_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(bins, 0, 256, s) != cudaSuccess) return GES_ERR_CUDA;
    BinArgs a;
    a.n = n;
    a.n_views = n_views;
    a.n_entries = (uint32_t)((uint64_t)n * n_views);
    a.rec = at<float4>(proj, PL.records);
    a.binrec = at<uint4>(proj, PL.binrec);
    a.total = at<unsigned long long>(proj, 0);
    a.err = at<uint32_t>(proj, 8);
    a.header = at<uint32_t>(bins, 0);
    for (int i = 0; i < 2; ++i) {
        a.dkey[i] = at<uint32_t>(bins, L.dkey[i]);
        a.dval[i] = at<uint32_t>(bins, L.dval[i]);
        a.ikey[i] = at<uint32_t>(bins, L.ikey[i]);
        a.ival[i] = at<uint32_t>(bins, L.ival[i]);
    }
    a.rcount = at<uint32_t>(bins, L.rcount);
    a.rinfo = at<uint4>(bins, L.rinfo);
    a.ranges = at<uint2>(bins, L.ranges);
    a.queue = at<uint32_t>(bins, L.queue);
    a.hist = at<uint32_t>(bins, L.hist);
    a.partials = at<uint32_t>(bins, L.partials);
    a.cap = cap;
    a.tile_bits = bits_for((uint32_t)V.n_tiles);
    a.build_queue = cfg->persistent != 0;
    a.V = V;
    return cuda_status(launch_bin(a, s));
}

ges_status ges_render_fwd(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                          const void *proj, size_t proj_bytes, const void *bins, size_t bins_bytes, float *color,
                          float *depth, float *alpha, float *normal, float *t_final, uint32_t *last,
                          uint32_t *n_contrib, uint32_t *n_eval, void *stream) {
    GES_RANGE();
    if (!check_views(n, n_views, cams, cfg) || !proj || !bins || !color || !alpha || !t_final || !last || !n_contrib)
        return GES_ERR_INVALID_ARG;
    const ProjLayout PL = proj_layout(n, n_views);
    if (proj_bytes < PL.bytes) return GES_ERR_INVALID_ARG;
    const ViewSet V = make_views(n_views, cams, cfg);
    const uint64_t cap = capacity_for(n, n_views, (uint32_t)V.n_tiles, bins_bytes);
    if (cap == UINT64_MAX) return GES_ERR_INVALID_ARG;
    const BinsLayout L = bins_layout(n, n_views, (uint32_t)V.n_tiles, cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FwdArgs a;
    a.rec = at<float4>(proj, PL.records);
    const int res = L.tile_passes & 1;
    a.inst_entry = at<uint32_t>(bins, L.ival[res]);
    a.ranges = at<uint2>(bins, L.ranges);
    a.queue = cfg->persistent ? at<uint32_t>(bins, L.queue) : nullptr;
    a.counter = const_cast<uint32_t *>(at<uint32_t>(bins, 4));
    a.color = color; a.depth = depth; a.alpha = alpha; a.normal = normal; a.t_final = t_final;
    a.last = last; a.n_contrib = n_contrib; a.n_eval = n_eval;
    a.n_events = n_eval ? const_cast<unsigned long long *>(at<unsigned long long>(bins, 16)) : nullptr;
    a.n_entries = (uint32_t)((uint64_t)n * n_views);
    a.err = const_cast<uint32_t *>(at<uint32_t>(proj, 8));
    a.batch = cfg->batch;
    a.alpha_min = cfg->alpha_min; a.alpha_max = cfg->alpha_max; a.t_min = cfg->t_min;
    for (int c = 0; c < 3; ++c) a.bg[c] = cfg->bg[c];
    a.V = V;
    if (a.queue && cudaMemsetAsync(a.counter, 0, 4, s) != cudaSuccess) return GES_ERR_CUDA;
    if (a.n_events && cudaMemsetAsync(a.n_events, 0, 8, s) != cudaSuccess) return GES_ERR_CUDA;
    return cuda_status(launch_render_fwd(a, s));
}

ges_status ges_render_bwd_screen(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                                 void *proj, size_t proj_bytes, const void *bins, size_t bins_bytes,
                                 const float *color, const float *depth, const float *normal, const float *t_final,
                                 const uint32_t *last, const float *g_color, const float *g_depth,
                                 const float *g_alpha, const float *g_normal, float *g2d, void *stream) {
    GES_RANGE();
    if (!check_views(n, n_views, cams, cfg) || !proj || !bins || !t_final || !last) return GES_ERR_INVALID_ARG;
    if ((g_color && !color) || (g_depth && !depth) || (g_normal && !normal)) return GES_ERR_INVALID_ARG;
    if (g2d && !aligned16(g2d)) return GES_ERR_INVALID_ARG;
    const ProjLayout PL = proj_layout(n, n_views);
    if (proj_bytes < PL.bytes) return GES_ERR_INVALID_ARG;
    const ViewSet V = make_views(n_views, cams, cfg);
    const uint64_t cap = capacity_for(n, n_views, (uint32_t)V.n_tiles, bins_bytes);
    if (cap == UINT64_MAX) return GES_ERR_INVALID_ARG;
    const BinsLayout L = bins_layout(n, n_views, (uint32_t)V.n_tiles, cap);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *acc = g2d ? g2d : at<float>(proj, PL.g2d);
    const size_t acc_bytes = (size_t)n * n_views * 64;
    if (acc_bytes && cudaMemsetAsync(acc, 0, acc_bytes, s) != cudaSuccess) return GES_ERR_CUDA;
    BwdArgs b;
    b.rec = at<float4>(proj, PL.records);
    const int res = L.tile_passes & 1;
    b.inst_entry = at<uint32_t>(bins, L.ival[res]);
    b.ranges = at<uint2>(bins, L.ranges);
    b.queue = cfg->persistent ? at<uint32_t>(bins, L.queue) : nullptr;
    b.counter = const_cast<uint32_t *>(at<uint32_t>(bins, 8));
    b.color = color; b.depth = depth; b.normal = normal; b.t_final = t_final; b.last = last;
    b.g_color = g_color; b.g_depth = g_depth; b.g_alpha = g_alpha; b.g_normal = g_normal;
    b.g2d = acc;
    b.n_entries = (uint32_t)((uint64_t)n * n_views);
    b.err = at<uint32_t>(proj, 8);
    b.batch = cfg->batch;
    b.alpha_min = cfg->alpha_min; b.alpha_max = cfg->alpha_max;
    b.V = V;
    if (b.queue && cudaMemsetAsync(b.counter, 0, 4, s) != cudaSuccess) return GES_ERR_CUDA;
    return cuda_status(launch_render_bwd(b, s));
}

// S8 for the splats [first, first + count) of n.
static ges_status preprocess_bwd_impl(int32_t n, int32_t first, int32_t count, int32_t n_views,
                                      const ges_camera *cams, const ges_config *cfg, const float *pos_op,
                                      const float *lscale_beta, const float *quat, const void *color_in,
                                      const void *proj, size_t proj_bytes, const float *g2d, float *g_pos_op,
                                      float *g_lscale_beta, float *g_quat, float *g_color_in, void *stream) {
    if (!check_views(n, n_views, cams, cfg) || !proj) return GES_ERR_INVALID_ARG;
    if (first < 0 || count < 0 || (int64_t)first + count > n) return GES_ERR_INVALID_ARG;
    if (n > 0 && (!pos_op || !lscale_beta || !quat || !color_in || !g_pos_op || !g_lscale_beta || !g_quat ||
                  !g_color_in || !aligned16(pos_op) || !aligned16(lscale_beta) || !aligned16(quat) ||
                  !aligned16(color_in) || !aligned16(g_pos_op) || !aligned16(g_lscale_beta) || !aligned16(g_quat)))
        return GES_ERR_INVALID_ARG;
    if (g2d && !aligned16(g2d)) return GES_ERR_INVALID_ARG;
    const ProjLayout PL = proj_layout(n, n_views);
    if (proj_bytes < PL.bytes) return GES_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PreBwdArgs p;
    p.n = n;
    p.first = first;
    p.count = count;
    p.pos_op = reinterpret_cast<const float4 *>(pos_op);
    p.lsb = reinterpret_cast<const float4 *>(lscale_beta);
    p.quat = reinterpret_cast<const float4 *>(quat);
    p.color = color_in;
    p.rec = at<float4>(proj, PL.records);
    p.g2d = reinterpret_cast<const float4 *>(g2d ? g2d : at<float>(proj, PL.g2d));
    p.g_pos_op = reinterpret_cast<float4 *>(g_pos_op);
    p.g_lsb = reinterpret_cast<float4 *>(g_lscale_beta);
    p.g_quat = reinterpret_cast<float4 *>(g_quat);
    p.g_color = g_color_in;
    p.P = make_params(cfg);
    p.V = make_views(n_views, cams, cfg);
    return cuda_status(launch_preprocess_bwd(p, s));
}

ges_status ges_preprocess_bwd(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                              const float *pos_op, const float *lscale_beta, const float *quat, const void *color_in,
                              const void *proj, size_t proj_bytes, const float *g2d, float *g_pos_op,
                              float *g_lscale_beta, float *g_quat, float *g_color_in, void *stream) {
    GES_RANGE();
    return preprocess_bwd_impl(n, 0, n, n_views, cams, cfg, pos_op, lscale_beta, quat, color_in, proj, proj_bytes,
                               g2d, g_pos_op, g_lscale_beta, g_quat, g_color_in, stream);
}

ges_status ges_preprocess_bwd_range(int32_t n, int32_t first, int32_t count, int32_t n_views,
                                    const ges_camera *cams, const ges_config *cfg, const float *pos_op,
                                    const float *lscale_beta, const float *quat, const void *color_in,
                                    const void *proj, size_t proj_bytes, const float *g2d, float *g_pos_op,
                                    float *g_lscale_beta, float *g_quat, float *g_color_in, void *stream) {
    GES_RANGE();
    return preprocess_bwd_impl(n, first, count, n_views, cams, cfg, pos_op, lscale_beta, quat, color_in, proj,
                               proj_bytes, g2d, g_pos_op, g_lscale_beta, g_quat, g_color_in, stream);
}

ges_status ges_render_bwd(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                          const float *pos_op, const float *lscale_beta, const float *quat, const void *color_in,
                          void *proj, size_t proj_bytes, const void *bins, size_t bins_bytes, const float *color,
                          const float *depth, const float *normal, const float *t_final, const uint32_t *last,
                          const float *g_color, const float *g_depth, const float *g_alpha, const float *g_normal,
                          float *g_pos_op, float *g_lscale_beta, float *g_quat, float *g_color_in, float *g2d,
                          void *stream) {
    GES_RANGE();
    // check both halves' arguments before launching either
    if (n > 0 && (!pos_op || !lscale_beta || !quat || !color_in || !g_pos_op || !g_lscale_beta || !g_quat ||
                  !g_color_in || !aligned16(pos_op) || !aligned16(lscale_beta) || !aligned16(quat) ||
                  !aligned16(g_pos_op) || !aligned16(g_lscale_beta) || !aligned16(g_quat)))
        return GES_ERR_INVALID_ARG;
    ges_status st = ges_render_bwd_screen(n, n_views, cams, cfg, proj, proj_bytes, bins, bins_bytes, color, depth,
                                          normal, t_final, last, g_color, g_depth, g_alpha, g_normal, g2d, stream);
    if (st != GES_OK) return st;
    return ges_preprocess_bwd(n, n_views, cams, cfg, pos_op, lscale_beta, quat, color_in, proj, proj_bytes, g2d,
                              g_pos_op, g_lscale_beta, g_quat, g_color_in, stream);
}

ges_status ges_sync_status(void *proj, size_t proj_bytes, void *stream) {
    GES_RANGE();
    if (!proj || proj_bytes < 256) return GES_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t word = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GES_ERR_CUDA;
    if (cudaMemcpyAsync(&word, static_cast<char *>(proj) + 8, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GES_ERR_CUDA;
    if (cudaMemsetAsync(static_cast<char *>(proj) + 8, 0, 4, s) != cudaSuccess) return GES_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GES_ERR_CUDA;
    if (word & kErrBounds) return GES_ERR_BOUNDS;
    if (word & kErrCapacity) return GES_ERR_CAPACITY;
    if (word & kErrNumeric) return GES_ERR_NUMERIC;
    return GES_OK;
}

}  // extern "C"
