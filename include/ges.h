/*
 * ges.h -- C ABI of libges.so, a GB300 (sm_103a) rasterizer for
 * generalized-exponential splats (GES), forward and backward.
 *
 * The method is the GES splatting of DyGASR (Sec. 3.2): each splat i has a
 * centre x_i, a covariance Sigma = R S S^T R^T (Eq. 4) whose scales are
 * modulated by phi(beta) (Eq. 6-7), a shape parameter beta (the paper's
 * epsilon, Eq. 1 and Eq. 3), an opacity and a colour. It is projected to the
 * image with Sigma' = J W Sigma W^T J^T (Sec. 3.2), evaluated with the falloff
 * exp(-1/2 Q^(beta/2)) of Eq. 3 (Q the Mahalanobis distance under Sigma'),
 * and composited front to back, the discrete form of the volume rendering
 * integral of Eq. 5, into colour, depth (Sec. 3.3, the depth map that mesh
 * extraction samples), alpha, and the normal n_g* of the flattened splats
 * (Sec. 3.3, Eq. 10-13). Beside the rasterizer: the reconstruction loss of Eq. 8
 * and its gradient (ges_loss_rgb), the 16-nearest-neighbour lists and the
 * generalized surface regularization of Eq. 9-13 at sample points (ges_knn,
 * ges_gsr), and the level-set points and normals of the mesh extraction of
 * Sec. 3.3 (ges_knn_points, ges_levelset).
 *
 * Conventions
 *  - Every pointer argument except `cams`, `cfg` and `count` is a DEVICE
 *    pointer owned by the caller. The library allocates nothing; it never calls
 *    cudaMalloc and never frees caller memory.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream), except ges_instance_count and ges_sync_status, which
 *    synchronise it.
 *  - Arguments are checked on the host before anything is launched; a bad
 *    argument returns GES_ERR_INVALID_ARG and launches nothing. A failed launch
 *    returns GES_ERR_CUDA. Conditions found on the device (instance capacity
 *    exceeded, non-finite projected values) are recorded in an error word inside
 *    `proj` and reported by ges_sync_status.
 *  - Arrays are float32 (the colour input may instead be 16-bit, see
 *    ges_config.color_storage), row-major, C-contiguous. All views of a call are
 *    concatenated: pixel arrays hold view 0's pixels, then view 1's, etc.
 *  - The calls are not thread-safe for one `proj` / `bins` pair; distinct
 *    buffers may be used concurrently on distinct streams.
 *
 * Readings where the paper is silent:
 *  - phi_mode 1 (default): phi(beta) = 2 / (1 + exp(-rho (beta - 2))), so
 *    phi(2) = 1 and beta = 2 is the 3DGS Gaussian; phi_mode 2 evaluates Eq. 7
 *    as printed, 2 / (1 + exp(-(rho beta - 2 beta))); phi_mode 0 is phi = 1.
 *    phi multiplies all three scales.
 *  - alpha = min(alpha_max, o exp(-1/2 Q^(beta/2))); alpha < alpha_min is
 *    skipped; the splat that would take transmittance below t_min ends the
 *    pixel and is not blended. The support used for binning is the exact level
 *    set Q <= q_cut = (2 ln(o / alpha_min))^(2 / beta).
 *  - Depth output = sum_i w_i z_i with z the camera-space z (not divided by
 *    alpha). Normal output = sum_i w_i n_i, n_i the world-space axis of the
 *    smallest scale turned to face the camera. Colour adds T_final * bg.
 *  - Colour: sh_degree -1 takes `color` as RGB [N, 3]; degree d in 0..3 takes
 *    real spherical-harmonic coefficients [N, (d+1)^2, 3] (Condon-Shortley
 *    phase, ordered by l then m = -l..l) evaluated in the direction from the
 *    camera centre to the splat, rgb = max(0, sum_k c_k Y_k + 0.5).
 *  - Pixel (x, y) is sampled at (x + 0.5, y + 0.5).
 *  - Depth order within a tile: ascending float32 camera depth
 *    z32 = ((r20 x + r21 y) + r22 z) + t2, each operation rounded to float32,
 *    ties by entry index (entry = view * N + splat). The same z32 decides the
 *    near-plane cull (z32 > znear).
 *  - Tile lists: tile t lists a splat iff the minimum of Q over the rectangle of
 *    pixel centres of t (clipped to the splat's pixel box) is <= q_cut (1 + 2^-10),
 *    evaluated in float32 without fused multiply-adds in a fixed operation order
 *    (edge minimisers use the correctly rounded reciprocals of the conic's a, c).
 */
#ifndef GES_H
#define GES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GES_API __attribute__((visibility("default")))
#else
#define GES_API
#endif

#define GES_ABI_VERSION 3
#define GES_MAX_VIEWS 32

typedef enum ges_status {
    GES_OK = 0,
    GES_ERR_INVALID_ARG = 1, /* host-side check failed; nothing was launched */
    GES_ERR_CAPACITY = 2,    /* more tile instances than `bins` holds; lists were truncated */
    GES_ERR_CUDA = 3,        /* a CUDA launch or copy failed */
    GES_ERR_NUMERIC = 4,     /* a splat had a non-finite position, opacity or beta, a beta <= 0, or (if
                                visible) a non-finite projection; it was culled */
    GES_ERR_TOO_LARGE = 5,   /* the problem exceeds the fixed scratch of ges_render_bwd_noalloc */
    GES_ERR_BOUNDS = 6       /* debug build only: a device-side bounds check failed; the access was
                                skipped (see ges_build_flags) */
} ges_status;

/* Pinhole camera. viewmat: row-major 3x4 world-to-camera [R | t]; camera x right,
 * y down, z forward. Pixel (x, y) maps to u = fx X/Z + cx, v = fy Y/Z + cy. */
typedef struct ges_camera {
    int32_t width, height;
    float fx, fy, cx, cy;
    float viewmat[12];
    float znear;
} ges_camera;

/* Rasterizer settings. Defaults (the "3DGS standards" the paper keeps, Sec. 4.2):
 * tile 16x16, batch 256, phi_mode 1, rho 0.1, lowpass 0.3, alpha_min 1/255,
 * alpha_max 0.99, t_min 1e-4, jac_clamp 1.3. */
typedef struct ges_config {
    int32_t tile_w, tile_h; /* 16x16, 16x8, 8x16, 8x8, 32x8 or 8x32 */
    int32_t batch;          /* render: list entries each warp prefetches ahead of the 32 it evaluates
                               (32..256, multiple of 32) */
    int32_t sh_degree;      /* -1 (RGB given) or 0..3 */
    int32_t phi_mode;       /* 0 off, 1 centred (default), 2 as printed in Eq. 7 */
    float rho;              /* shape strength of Eq. 7 (0.1, Sec. 4.2) */
    float lowpass;          /* h added to the diagonal of Sigma' */
    float alpha_min, alpha_max, t_min;
    float jac_clamp;        /* |X/Z| is clamped to jac_clamp * (W/2)/fx in J (likewise y) */
    float bg[3];            /* background colour */
    int32_t persistent;     /* 0: one CTA per tile; 1: persistent warps taking (tile, 8x4 block) items of a
                               longest-first tile queue */
    int32_t color_storage;  /* element type of the colour input (`color` of ges_preprocess, `color_in` of the
                               backward calls): 0 float32, 1 IEEE binary16, 2 bfloat16. The values are widened
                               to float32 on load and everything after is float32; gradients stay float32 */
} ges_config;

/* Number of bytes `proj` must hold for n splats and n_views views:
 * per (view, splat) a 64-byte render record, a 32-byte binning record and a
 * 64-byte screen-space gradient accumulator, plus a 256-byte header. */
GES_API size_t ges_proj_bytes(int32_t n, int32_t n_views);

/* Number of bytes `bins` must hold to bin up to `capacity` tile instances
 * (splat-tile overlaps) for n splats over the given views and tile shape. */
GES_API size_t ges_bins_bytes(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                      uint64_t capacity);

/* S1-S4: projection (Eq. 4, Eq. 6-7, Sec. 3.2), GES support (Eq. 3), colour and
 * normal, tile counts and float32 depth keys, for every (view, splat) entry.
 * Inputs (device, float32):
 *   pos_op      [n, 4]  x, y, z, opacity in (0, 1] (already activated)
 *   lscale_beta [n, 4]  log-scales l1, l2, l3 and beta > 0
 *   quat        [n, 4]  rotation (w, x, y, z), any non-zero norm
 *   color       [n, 3] RGB (sh_degree -1) or [n, (d+1)^2, 3] SH coefficients, float32 or the
 *               16-bit type cfg->color_storage names; 16-byte aligned
 * cams: host array of n_views cameras (1 <= n_views <= GES_MAX_VIEWS).
 * Writes `proj` (ges_proj_bytes(n, n_views) bytes, 16-byte aligned), and the
 * total instance count read by ges_instance_count. Clears the error word. */
GES_API ges_status ges_preprocess(int32_t n, const float *pos_op, const float *lscale_beta, const float *quat,
                          const void *color, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                          void *proj, size_t proj_bytes, void *stream);

/* ges_preprocess for the splats [first, first + count) of the n only (their entries in
 * every view; the pointers are those of all n splats). The call whose range starts at 0
 * clears the instance total and the error word, so it goes first; the ranges of one step
 * must not overlap and must cover [0, n) before ges_bin. This lets a caller start on the
 * first splats while the later ones are still being copied to the device. */
GES_API ges_status ges_preprocess_range(int32_t n, int32_t first, int32_t count, const float *pos_op,
                                        const float *lscale_beta, const float *quat, const void *color,
                                        int32_t n_views, const ges_camera *cams, const ges_config *cfg, void *proj,
                                        size_t proj_bytes, void *stream);

/* Synchronises `stream` and returns in *count the number of tile instances that
 * the last ges_preprocess on `proj` produced (sum of tiles touched). */
GES_API ges_status ges_instance_count(const void *proj, size_t proj_bytes, uint64_t *count, void *stream);

/* S5: binning. Sorts entries by float32 depth (stable LSD radix sort), emits one
 * (global tile, entry) instance per listed tile in depth order, sorts the
 * instances by tile (stable, so depth order is kept within a tile) and finds
 * each tile's [start, end) range. With cfg->persistent it also builds the
 * longest-first tile queue. If the instances exceed the capacity `bins` was
 * sized for, the lists are truncated and GES_ERR_CAPACITY is recorded. */
GES_API ges_status ges_bin(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg, void *proj,
                   size_t proj_bytes, void *bins, size_t bins_bytes, void *stream);

/* S6: forward compositing (Eq. 3 falloff, Eq. 5 discretised). Outputs, for the
 * concatenated views (P = sum of width*height):
 *   color   [3 per view, planar]: view v occupies 3*W_v*H_v floats, channel-major
 *   depth   [P]  sum_i w_i z_i
 *   alpha   [P]  1 - T_final
 *   normal  [like color]  sum_i w_i n_i
 *   t_final [P]  final transmittance
 *   last    [P]  one past the sorted-instance index of the last blended splat
 *                (the tile's start if none): the backward replays [start, last)
 *   n_contrib [P] number of blended splats
 *   n_eval  [P]  number of tile-list entries the pixel evaluated before it ended
 *                (the work count of the pixel; used for roofline accounting). When
 *                n_eval is given, the call also stores at byte 16 of `bins` (uint64)
 *                the number of (8x4 pixel block, splat) pairs that passed the warp's
 *                support cull, i.e. the pairs its warps evaluated 32 pixels at a time
 * depth, normal and n_eval may be NULL (not written); with neither depth nor normal (a
 * render for a loss on the colour, as in training) their accumulations are left out. */
GES_API ges_status ges_render_fwd(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                                  const void *proj, size_t proj_bytes, const void *bins, size_t bins_bytes,
                                  float *color, float *depth, float *alpha, float *normal, float *t_final,
                                  uint32_t *last, uint32_t *n_contrib, uint32_t *n_eval, void *stream);

/* S7 + S8: backward. Replays the forward front to back from t_final and last
 * (no per-pixel lists are stored): with w_i = alpha_i T_i and X a final output,
 * dX/dalpha_i = T_i x_i - (X - sum_{j<=i} w_j x_j) / (1 - alpha_i), and for the
 * alpha output T_final / (1 - alpha_i). Per-splat screen-space gradients are
 * summed across each warp before FP32 atomics into a per-entry accumulator
 * (g2d, 16 floats per entry: dL/du, dL/dv; dL/dSigma' as the symmetric-matrix
 * gradient G00, G01, G11 (dL = G00 dS00 + 2 G01 dS01 + G11 dS11); opacity, beta,
 * z, r, g, b, -, nx, ny, nz, -), which the chain rule of S1-S4 then takes back
 * to the inputs.
 * Inputs: the forward's inputs, `proj`/`bins` as left by ges_bin, the forward's
 * color, depth, normal, t_final and last, and the upstream gradients (same
 * layouts as the outputs; any of g_color, g_depth, g_alpha, g_normal may be NULL
 * for zero). Outputs g_pos_op, g_lscale_beta, g_quat, g_color_in have the input
 * layouts (g_color_in in float32 whatever cfg->color_storage) and are OVERWRITTEN
 * (summed over views). Without g_depth and g_normal (a loss on the colour, as in
 * training) the replay leaves out the depth and normal channels, which is faster. g2d may be NULL, else it
 * receives the per-entry screen-space gradients [n_views * n, 16]. */
GES_API ges_status ges_render_bwd(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                          const float *pos_op, const float *lscale_beta, const float *quat, const void *color_in,
                          void *proj, size_t proj_bytes, const void *bins, size_t bins_bytes,
                          const float *color, const float *depth, const float *normal, const float *t_final,
                          const uint32_t *last, const float *g_color, const float *g_depth,
                          const float *g_alpha, const float *g_normal, float *g_pos_op, float *g_lscale_beta,
                          float *g_quat, float *g_color_in, float *g2d, void *stream);

/* The two halves of ges_render_bwd, for callers that schedule or time them
 * separately. ges_render_bwd_screen is S7 alone: it zeroes the accumulator (g2d,
 * or the one inside `proj` if g2d is NULL) and sums every pixel's screen-space
 * gradient into it. ges_preprocess_bwd is S8 alone: it takes that accumulator
 * (g2d, or the one inside `proj` if NULL) back to the 3-D inputs (overwriting
 * g_pos_op, g_lscale_beta, g_quat, g_color_in). Arguments are as for
 * ges_render_bwd. */
GES_API ges_status ges_render_bwd_screen(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                                         void *proj, size_t proj_bytes, const void *bins, size_t bins_bytes,
                                         const float *color, const float *depth, const float *normal,
                                         const float *t_final, const uint32_t *last, const float *g_color,
                                         const float *g_depth, const float *g_alpha, const float *g_normal,
                                         float *g2d, void *stream);

GES_API ges_status ges_preprocess_bwd(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                                      const float *pos_op, const float *lscale_beta, const float *quat,
                                      const void *color_in, const void *proj, size_t proj_bytes, const float *g2d,
                                      float *g_pos_op, float *g_lscale_beta, float *g_quat, float *g_color_in,
                                      void *stream);

/* ges_preprocess_bwd for the splats [first, first + count) of the n only: their rows of
 * g_pos_op, g_lscale_beta, g_quat and g_color_in are written, the others left as they are
 * (so a caller can copy finished rows back to the host while later ranges run). */
GES_API ges_status ges_preprocess_bwd_range(int32_t n, int32_t first, int32_t count, int32_t n_views,
                                            const ges_camera *cams, const ges_config *cfg, const float *pos_op,
                                            const float *lscale_beta, const float *quat, const void *color_in,
                                            const void *proj, size_t proj_bytes, const float *g2d, float *g_pos_op,
                                            float *g_lscale_beta, float *g_quat, float *g_color_in, void *stream);

/* ges_render_bwd for callers that cannot allocate device memory.
 *
 * The paper has no counterpart to this call; it is a property of the library.
 * ges_render_bwd needs an accumulator of 16 floats per (view, splat) entry that
 * the caller provides (inside `proj`, or as `g2d`). Callers that must not
 * allocate while they run (cudaMalloc can synchronise the device and has no
 * bounded latency, so interactive and real-time loops avoid it; some host
 * applications also keep all device memory in their own pool and hand a library
 * only the tensors it reads and writes) can call this variant instead. It
 * computes the same gradients, with the accumulator in a fixed array inside the
 * library, so it allocates nothing and needs no scratch from the caller.
 *
 * Arguments: as ges_render_bwd, without g2d. `proj` must still be the buffer
 * ges_preprocess filled (its own accumulator region is not used).
 * Limit: n * n_views <= GES_NOALLOC_MAX_ENTRIES (524,288 entries, a 32 MiB array
 * that every GPU which loads the library keeps until the process exits); larger
 * problems return GES_ERR_TOO_LARGE and launch nothing.
 * Set-up: the first call on a device (with that device current) looks up the
 * array's device address; make that first call before any stream capture. The
 * address is kept for the life of the process: after cudaDeviceReset the
 * library's device code is loaded again, possibly elsewhere, so a process that
 * resets a device must not call this entry point on it again.
 * Sharing: all calls use the same array, which keeps the previous call's
 * contents; each call zeroes the part it uses on `stream` before accumulating.
 * Calls that overlap on the GPU (different streams, or different threads on the
 * same device) race on the array and give wrong gradients. */
#define GES_NOALLOC_MAX_ENTRIES 524288
GES_API ges_status ges_render_bwd_noalloc(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                                          const float *pos_op, const float *lscale_beta, const float *quat,
                                          const void *color_in, void *proj, size_t proj_bytes, const void *bins,
                                          size_t bins_bytes, const float *color, const float *depth,
                                          const float *normal, const float *t_final, const uint32_t *last,
                                          const float *g_color, const float *g_depth, const float *g_alpha,
                                          const float *g_normal, float *g_pos_op, float *g_lscale_beta,
                                          float *g_quat, float *g_color_in, void *stream);

/* Byte offsets of the arrays inside `proj` and `bins`, for callers that inspect
 * the intermediate results (tests, tools). Host-only; launches nothing.
 *   proj.records  [n_views * n] x 16 float: (u, v, a, b), (c, q_cut, beta/2, o),
 *                 (r, g, b, z), (nx, ny, nz, 0); entry e = view * n + splat
 *   proj.binrec   [n_views * n] x 8 x 32-bit: ext_x, ext_y (float), tiles touched,
 *                 z32 bits (uint32; 0xffffffff if not listed), hit mask over the
 *                 tile box (row-major; valid when the box has <= 32 tiles), box
 *                 origin tx0 | ty0 << 16, box size w | h << 16, 0
 *   proj.g2d      [n_views * n] x 16 float screen-space gradient accumulator (see
 *                 ges_render_bwd for the layout)
 *   bins.inst_tile / inst_entry  [n_instances] uint32, sorted by (tile, z32, entry)
 *   bins.ranges   [n_tiles] x 2 uint32 [start, end) per global tile (0, 0 if empty);
 *                 global tile = tile_base[view] + ty * tiles_x + tx
 *   bins.queue    [n_tiles] uint32 global tile ids, longest list first          */
typedef struct ges_layout {
    uint64_t proj_records, proj_binrec, proj_g2d, proj_bytes;
    uint64_t bins_inst_tile, bins_inst_entry, bins_ranges, bins_queue, bins_bytes;
    uint32_t n_tiles;
    uint32_t tile_base[GES_MAX_VIEWS];
} ges_layout;

GES_API ges_status ges_get_layout(int32_t n, int32_t n_views, const ges_camera *cams, const ges_config *cfg,
                          uint64_t capacity, ges_layout *out);

/* ---------------------------------------------------------------- loss
 * Reconstruction loss of Eq. 8 (Sec. 3.2), L_rgb = (1 - lambda) L_1 + lambda L_SSIM,
 * per view, and its gradient with respect to the rendered colour, which is the
 * g_color that ges_render_bwd takes. Readings (the paper names the terms only):
 * L_1 = mean over pixels and the 3 channels of |C - C_target|; L_SSIM = 1 - mean
 * over pixels and channels of the SSIM map of Wang et al. (2004) with an 11 x 11
 * Gaussian window of standard deviation 1.5 (normalised), C1 = 0.01^2, C2 = 0.03^2,
 * both images taken as 0 outside the frame (zero padding), the map evaluated at
 * every pixel. Each view has its own loss; dL_rgb(v)/dC_v is that view's gradient.
 *
 * Workspace: ges_loss_workspace_bytes(n_views, cams) bytes of device memory (per-CTA
 * partial sums; contents need not be initialised; not shared by concurrent calls).
 *   color, target  [3 * sum_v W_v H_v] planar per view, the layout of ges_render_fwd's
 *                  color (target values are taken as given; no clamping)
 *   lambda         weight of L_SSIM, in [0, 1] (the paper: 0.2)
 *   loss           [n_views] float32, L_rgb of each view (written)
 *   g_color        [like color] float32, dL_rgb(v)/dC (written); NULL: loss only
 * The sums are formed in a fixed order (no atomics), so results are reproducible. */
GES_API size_t ges_loss_workspace_bytes(int32_t n_views, const ges_camera *cams);

/* ---------------------------------------------------------------- KNN (GSR neighbours)
 * The GES_KNN_K = 16 splat centres nearest to each splat centre (Euclidean, the
 * splat itself included), for the density of the generalized surface regularization
 * (Sec. 3.3, Eq. 9; the paper sums over the 16 closest points, Sec. 4.2).
 *   pos_op   [n, 4] float32 (x, y, z, opacity), 16-byte aligned; opacity unused
 *   knn      [n, 16] int32 (written): splat i's neighbours by increasing distance,
 *            ties to the lower index (so neighbour 0 is i itself unless another centre
 *            coincides with it and has a lower index)
 * Exact (distances are squared float32 differences summed in x, y, z order) unless
 * one query must examine more than 65,536 candidate centres (tens of thousands of
 * coincident centres, or non-finite coordinates); its list is then the best among
 * those examined. Workspace: ges_knn_workspace_bytes(n) bytes, 256-byte aligned, no
 * initialisation needed. n must be in [16, 2^26]; otherwise both calls reject it
 * (0 / GES_ERR_INVALID_ARG). */
#define GES_KNN_K 16
GES_API size_t ges_knn_workspace_bytes(int32_t n);
GES_API ges_status ges_knn(int32_t n, const float *pos_op, void *workspace, size_t workspace_bytes, int32_t *knn,
                           void *stream);

/* The GES_KNN_K splat centres nearest to each of m arbitrary points, for the density
 * along a level-set ray (Sec. 3.3, "Mesh Extraction": the start point's 16 closest
 * splats, as in Sec. 4.2); ges_levelset calls the same search.
 *   points   [m, 4] float32 (x, y, z, w), 16-byte aligned; w = 0 marks a point without a
 *            query (its list is all -1)
 *   knn      [m, 16] int32 (written, 16-byte aligned): point j's neighbours by increasing
 *            distance, ties to the lower index
 * The points are searched in grid-cell order; cells are grouped in 2 x 2 x 2 blocks whose
 * counts let a query in empty space skip them. Exactness and the 65,536-candidate bound
 * are as for ges_knn. Workspace: ges_knn_points_workspace_bytes(n, m) bytes, 256-byte
 * aligned, no initialisation needed. n in [16, 2^26], m in [1, 2^28]. */
GES_API size_t ges_knn_points_workspace_bytes(int32_t n, int32_t m);
GES_API ges_status ges_knn_points(int32_t n, const float *pos_op, int32_t m, const float *points, void *workspace,
                                  size_t workspace_bytes, int32_t *knn, void *stream);

/* ---------------------------------------------------------------- GSR point evaluation
 * Generalized surface regularization at m sample points (Sec. 3.3): the density of
 * Eq. 9 over the GES_KNN_K splats nearest to the splat a sample was drawn from, the
 * ideal flat density of Eq. 10, the SDFs of Eq. 11, L_sdf (Eq. 12), L_nor (Eq. 13),
 * and the gradient of lambda_sdf L_sdf + lambda_nor L_nor (the weights of Eq. 14 are
 * the caller's; the paper does not give them). Readings (the paper gives the
 * equations only):
 *  - sample k is x = mu_j + R_j (s'_j * z_k), j = sample_splat[k], z_k ~ N(0, I) given
 *    (sample_z [m, 3]); gradients flow through x to splat j;
 *  - its neighbours are knn[j] (ges_knn: the 16 centres nearest to splat j, j included);
 *  - d = sum_i o_i exp(-1/2 P_i), P_i = Q_i^(beta_i/2), Q_i the Mahalanobis distance
 *    under Sigma_i = R_i diag(s'_i^2) R_i^T, s' = phi(beta) exp(l) (cfg->phi_mode and
 *    cfg->rho as in the rasterizer; the other fields of cfg are not used);
 *  - g* = the neighbour with the largest exp(-1/2 P_i), i.e. the smallest P_i (ties: the
 *    earlier one); n* = g*'s smallest-scale axis turned so that e = <x - mu*, n*> >= 0;
 *    s_min = g*'s smallest s'; ideal density dbar = exp(-1/2 (e^2 / s_min^2)^(beta* / 2));
 *  - f = s_min sqrt(-2 ln d) with d clamped to [1e-30, 1], fbar = s_min sqrt(-2 ln dbar);
 *  - L_sdf = mean |fbar - f|; L_nor = mean |u - n*|^2 with u the direction of grad f,
 *    i.e. of -grad d, summed relative to its largest term so that it stays defined
 *    where d underflows.
 * Inputs as for ges_preprocess; knn [n, 16] int32 (entries outside [0, n) are skipped);
 * sample_splat [m] int32 (samples outside [0, n) contribute nothing, but count in m).
 * Outputs: losses [3] float32 (L_sdf, L_nor, lambda_sdf L_sdf + lambda_nor L_nor);
 * sample_out [m, 8] float32 or NULL: x, y, z, d, f, fbar, u . n*, g*'s neighbour slot;
 * g_pos_op, g_lscale_beta, g_quat [n, 4] float32 (written, not accumulated), or all
 * three NULL for the losses only. Workspace: ges_gsr_workspace_bytes(n, m) bytes,
 * 256-byte aligned, no initialisation needed. Gradient sums use float atomics, so
 * their last bits vary from run to run; the losses are summed in a fixed order. */
/* ---------------------------------------------------------------- level-set points
 * Isosurface points with normals from rendered depth (Sec. 3.3, "Mesh Extraction"; the
 * paper's level is 0.3, Sec. 4.2), the input of a Poisson reconstruction. For each of the
 * m sampled pixels (pixels [m, 2] int32: view, pixel index y * W + x):
 *  - x0 = the point on the ray through the pixel centre at camera depth D / A, with D and
 *    A the pixel's rendered depth and alpha (depth, alpha: ges_render_fwd's outputs, all
 *    views concatenated); pixels with A < 1e-4, a non-finite x0, a view outside 0..n_views-1
 *    or an index outside their view give no point. v = the ray's unit direction.
 *  - the density of Eq. 9 along the ray is summed over the GES_KNN_K splats whose centres
 *    are nearest to x0 (the same 16 for the whole ray);
 *  - g = the one of them with the largest falloff at x0; the ray is sampled at n_steps
 *    (2..1024) evenly spaced t in [-3 sigma, 3 sigma], sigma^2 = v^T Sigma_g v;
 *  - the point is the first crossing from the camera side, d(t_k) < level <= d(t_k+1),
 *    linearly interpolated; the normal is grad f / |grad f| there (the direction of
 *    -grad d, summed relative to its largest term).
 * points [m, 8] float32 (written): x, y, z, nx, ny, nz, t, valid (1 or 0; the other
 * fields are 0 when there is no point). cfg: phi_mode and rho as in the rasterizer.
 * Workspace: ges_levelset_workspace_bytes(n, m) bytes, 256-byte aligned, no
 * initialisation needed. */
GES_API size_t ges_levelset_workspace_bytes(int32_t n, int32_t m);
GES_API ges_status ges_levelset(int32_t n, const float *pos_op, const float *lscale_beta, const float *quat,
                                const ges_config *cfg, int32_t n_views, const ges_camera *cams, const float *depth,
                                const float *alpha, int32_t m, const int32_t *pixels, int32_t n_steps, float level,
                                void *workspace, size_t workspace_bytes, float *points, void *stream);

GES_API size_t ges_gsr_workspace_bytes(int32_t n, int32_t m);
GES_API ges_status ges_gsr(int32_t n, const float *pos_op, const float *lscale_beta, const float *quat,
                           const ges_config *cfg, const int32_t *knn, int32_t m, const int32_t *sample_splat,
                           const float *sample_z, float lambda_sdf, float lambda_nor, void *workspace,
                           size_t workspace_bytes, float *losses, float *sample_out, float *g_pos_op,
                           float *g_lscale_beta, float *g_quat, void *stream);
GES_API ges_status ges_loss_rgb(int32_t n_views, const ges_camera *cams, const float *color, const float *target,
                                float lambda, void *workspace, size_t workspace_bytes, float *loss, float *g_color,
                                void *stream);

/* Synchronises `stream`, reads and clears the device error word in `proj`, and
 * returns the first recorded condition (GES_OK if none). */
GES_API ges_status ges_sync_status(void *proj, size_t proj_bytes, void *stream);

/* Static description of a status code. */
GES_API const char *ges_status_string(ges_status s);

/* ---------------------------------------------------------------- measurement
 * Throughput microbenchmarks for the roofline denominators of the issue-bound
 * kernels (a measurement utility; the paper has no counterpart). One kernel is
 * launched on `stream`, blocks_per_sm (1..64) CTAs of 256 threads per SM:
 *   kind 0  FP32 fused multiply-add, 8 independent chains per thread;
 *           *ops = flops (an FMA counts two)
 *   kind 1  ex2.approx (special-function unit), 8 chains per thread; *ops = ex2
 *   kind 2  rcp.approx (special-function unit), 8 chains per thread; *ops = rcp
 *   kind 3  FP32 atomic adds: each warp adds into `iters` 64-byte lines of
 *           `sink` chosen by a hash, 16 lanes per line and instruction (the
 *           render backward's accumulator update); *ops = atomic adds
 * iters: loop trips per thread (kinds 0-2, 16 operations per chain and trip)
 * or per warp (kind 3). sink: device buffer of sink_floats floats
 * (>= 256; for kind 3 a multiple of 16, its lines are the targets and are
 * modified). *ops (host) receives the operations the launch performs; time the
 * launch with events on `stream`. */
GES_API ges_status ges_peak_run(int32_t kind, int32_t blocks_per_sm, int32_t iters, float *sink,
                                uint64_t sink_floats, void *stream, uint64_t *ops);

/* Build flags of the loaded library: bit 0 set in the debug build (compiled with GES_DEBUG),
 * whose render kernels check every list entry they read against the number of (view, splat)
 * entries, and every pixel's replay end against its tile's list, before they use it: a failed
 * check records GES_ERR_BOUNDS in the error word (ges_sync_status) and skips the access instead
 * of faulting. The release build has no such checks. */
#define GES_BUILD_DEBUG 1
GES_API int32_t ges_build_flags(void);

/* GES_ABI_VERSION of the loaded library. */
GES_API int32_t ges_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GES_H */
