// Backward pass for callers that cannot allocate device memory.
//
// ges_render_bwd adds every pixel's per-splat screen-space gradient into an
// accumulator of 16 floats per (view, splat) entry, and that accumulator is
// memory the caller hands in (inside `proj`, or a separate `g2d` buffer). Some
// callers have no way to supply such extra memory: programs that must not call
// cudaMalloc once they run, because it can synchronise the whole device and has
// no bound on how long it takes (interactive or real-time loops), and host
// applications that reserve the device's memory for their own allocator and
// pass a library only the tensors it reads and writes.
//
// ges_render_bwd_noalloc serves them: it runs the same backward with the
// accumulator placed in a fixed array inside this library, so the caller passes
// inputs and outputs only. The array holds GES_NOALLOC_MAX_ENTRIES entries
// (32 MiB) and stays resident on every GPU that loads the library until the
// process exits.
#include <mutex>

#include "ges_internal.cuh"

namespace {

constexpr uint64_t kMaxEntries = GES_NOALLOC_MAX_ENTRIES;

// The accumulator. In host code this name stands for the symbol, not for a
// device address; host code asks the runtime for the address (below) and passes
// that to the kernels.
static __device__ __align__(256) float g_accumulator[kMaxEntries * 16];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float *g_accumulator_addr[kMaxDevices] = {};

// Device address of the accumulator on the current device, looked up once per
// device (with that device current) and cached.
ges_status accumulator_address(float **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GES_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_accumulator_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_accumulator) != cudaSuccess || !p) return GES_ERR_CUDA;
        g_accumulator_addr[dev] = static_cast<float *>(p);
    }
    *out = g_accumulator_addr[dev];
    return GES_OK;
}

}  // namespace

extern "C" ges_status ges_render_bwd_noalloc(
    int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg, const float *pos_op,
    const float *lscale_beta, const float *quat, const void *color_in, void *proj, size_t proj_bytes,
    const void *bins, size_t bins_bytes, const float *color, const float *depth, const float *normal,
    const float *t_final, const uint32_t *last, const float *g_color, const float *g_depth, const float *g_alpha,
    const float *g_normal, float *g_pos_op, float *g_lscale_beta, float *g_quat, float *g_color_in, void *stream) {
    GES_RANGE();
    if (n < 0 || n_views < 1) return GES_ERR_INVALID_ARG;
    if ((uint64_t)n * (uint64_t)n_views > kMaxEntries) return GES_ERR_TOO_LARGE;
    float *acc = nullptr;
    const ges_status st = accumulator_address(&acc);
    if (st != GES_OK) return st;
    // The accumulator keeps the previous call's sums; ges_render_bwd zeroes the
    // first n * n_views entries on `stream` before it accumulates.
    return ges_render_bwd(n, n_views, cams, cfg, pos_op, lscale_beta, quat, color_in, proj, proj_bytes, bins,
                          bins_bytes, color, depth, normal, t_final, last, g_color, g_depth, g_alpha, g_normal,
                          g_pos_op, g_lscale_beta, g_quat, g_color_in, acc, stream);
}
