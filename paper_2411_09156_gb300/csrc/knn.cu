// Exact k = 16 nearest splat centres (Sec. 4.2: the GSR density at a sample uses
// the 16 splats closest to the splat it was drawn from).
//
// A uniform grid over the centres' bounding box, at most two cells per point, is
// built on the device: cell keys, a stable radix sort of the points by cell (the
// sort of the binning), dense cell ranges and a cell-ordered copy of the centres.
// Each query then walks Chebyshev rings of cells around its own cell, keeping its 16
// best (distance, index) pairs sorted in registers, and stops once the 16th best
// distance is within the distance from the query to the part of the grid's box outside
// the searched block (no unsearched point can be closer). Once it holds 16, rows and
// cells whose box lies farther than the 16th are skipped without reading their ranges,
// which keeps queries away from the centres (points in front of a surface) from reading
// every cell of their block. Queries run in cell order, so a warp searches one
// neighbourhood. Distances are squared float32 with a fixed operation order; ties go to
// the lower index. A query examines at most 65,536 candidates (a bound that well-spread
// centres never reach; tens of thousands of coincident centres would), so no input makes
// the search quadratic.
#include "ges_internal.cuh"

namespace ges {

namespace {

constexpr int kK = GES_KNN_K;
constexpr uint32_t kQueryBudget = 1u << 16;  // candidate points one query may examine

struct KnnGrid {
    float lo[3];
    float h, inv_h;
    int dims[3];
    float slack;  // bound on how far float32 rounding can put a point outside its cell's box
};

struct KnnLayout {
    uint64_t bbox, grid, keys0, keys1, vals0, vals1, hist, partials, ranges, bcount, spos, bytes;
    uint32_t cap_cells, nblocks;
    int bits;
};

inline uint64_t al256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

KnnLayout knn_layout(int32_t n) {
    KnnLayout L;
    uint64_t cap = 2ull * (uint64_t)n;
    if (cap < 1) cap = 1;
    if (cap > (1ull << 27)) cap = 1ull << 27;
    L.cap_cells = (uint32_t)cap;
    L.bits = 1;
    while ((1ull << L.bits) < cap) ++L.bits;
    L.nblocks = ceil_div_u64(n > 0 ? (uint64_t)n : 1, kSortTile);
    uint64_t off = 0;
    L.bbox = off; off = al256(off + 6 * 4);
    L.grid = off; off = al256(off + sizeof(KnnGrid));
    L.keys0 = off; off = al256(off + 4ull * n);
    L.keys1 = off; off = al256(off + 4ull * n);
    L.vals0 = off; off = al256(off + 4ull * n);
    L.vals1 = off; off = al256(off + 4ull * n);
    L.hist = off; off = al256(off + 4ull * 256 * L.nblocks);
    L.partials = off; off = al256(off + 4ull * (ceil_div_u64(256ull * L.nblocks, kScanTile) + 1));
    L.ranges = off; off = al256(off + 8ull * L.cap_cells);
    L.bcount = off; off = al256(off + 4ull * L.cap_cells);  // blocks <= cells <= cap_cells
    L.spos = off; off = al256(off + 16ull * n);
    L.bytes = off;
    return L;
}

// float <-> order-preserving uint32 (for atomic min / max)
__device__ __forceinline__ uint32_t f2ord(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__global__ void __launch_bounds__(256) k_knn_bbox(const float4 *pos, int n, uint32_t *bb) {
    uint32_t mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, mx[3] = {0u, 0u, 0u};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = __ldg(pos + i);
        const float c[3] = {p.x, p.y, p.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint32_t o = f2ord(c[k]);
            mn[k] = min(mn[k], o);
            mx[k] = max(mx[k], o);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        mn[k] = __reduce_min_sync(0xffffffffu, mn[k]);
        mx[k] = __reduce_max_sync(0xffffffffu, mx[k]);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(bb + k, mn[k]);
            atomicMax(bb + 3 + k, mx[k]);
        }
    }
}

// Cell size h with at most cap cells: start from the volume per cell, then grow h
// until the product of the per-axis counts fits (flat boxes have a zero extent).
__global__ void k_knn_grid(const uint32_t *bb, uint32_t cap, KnnGrid *g) {
    float lo[3], ext[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = ord2f(bb[k]);
        ext[k] = fmaxf(ord2f(bb[3 + k]) - lo[k], 0.f);
    }
    const float emax = fmaxf(fmaxf(ext[0], ext[1]), ext[2]);
    float h = emax > 0.f ? emax : 1.f;
    const double vol = (double)fmaxf(ext[0], 1e-30f) * fmaxf(ext[1], 1e-30f) * fmaxf(ext[2], 1e-30f);
    const double h0 = cbrt(vol / (double)cap);
    if (h0 > 0.0 && h0 < (double)h) h = (float)h0;
    int d[3] = {1, 1, 1};
    bool fits = false;
    for (int it = 0; it < 256 && !fits; ++it) {
        double prod = 1.0;
        for (int k = 0; k < 3; ++k) {
            d[k] = (int)fminf(fmaxf(floorf(ext[k] / h) + 1.f, 1.f), 2048.f);
            prod *= d[k];
        }
        fits = prod <= (double)cap;
        if (!fits) h *= 1.0625f;
    }
    if (!fits || !(h > 0.f) || !isfinite(h)) {  // non-finite coordinates: one cell (the query budget bounds the work)
        d[0] = d[1] = d[2] = 1;
        h = 1.f;
    }
    for (int k = 0; k < 3; ++k) {
        g->lo[k] = isfinite(lo[k]) ? lo[k] : 0.f;
        g->dims[k] = d[k];
    }
    g->h = h;
    g->inv_h = 1.f / h;
    float amax = 0.f;
    for (int k = 0; k < 3; ++k) amax = fmaxf(amax, fabsf(g->lo[k]) + (float)d[k] * h);
    g->slack = 4e-6f * amax;
}

__device__ __forceinline__ int cell_axis(float p, float lo, float inv_h, int dim) {
    const int c = (int)floorf((p - lo) * inv_h);
    return min(max(c, 0), dim - 1);
}

// Blocks of 2 x 2 x 2 cells, with their point counts, let point queries skip empty space.
__device__ __forceinline__ int block_dim(int d) { return (d + 1) >> 1; }

__global__ void __launch_bounds__(256) k_knn_keys(const float4 *pos, int n, const KnnGrid *g, uint32_t *keys,
                                                  uint32_t *bcount) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 p = __ldg(pos + i);
    const KnnGrid G = *g;
    const int cx = cell_axis(p.x, G.lo[0], G.inv_h, G.dims[0]);
    const int cy = cell_axis(p.y, G.lo[1], G.inv_h, G.dims[1]);
    const int cz = cell_axis(p.z, G.lo[2], G.inv_h, G.dims[2]);
    keys[i] = (uint32_t)(cx + G.dims[0] * (cy + G.dims[1] * cz));
    atomicAdd(bcount + ((cx >> 1) + block_dim(G.dims[0]) * ((cy >> 1) + block_dim(G.dims[1]) * (cz >> 1))), 1u);
}

__global__ void __launch_bounds__(256) k_knn_ranges(const uint32_t *keys, const uint32_t *idx, const float4 *pos,
                                                    int n, uint2 *ranges, float4 *spos) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t k = keys[r];
    if (r == 0 || keys[r - 1] != k) ranges[k].x = (uint32_t)r;
    if (r == n - 1 || keys[r + 1] != k) ranges[k].y = (uint32_t)r + 1;
    const uint32_t i = idx[r];
    const float4 p = __ldg(pos + i);
    spos[r] = make_float4(p.x, p.y, p.z, __uint_as_float(i));
}

__device__ __forceinline__ float dist2(float4 a, float4 b) {
    const float dx = __fsub_rn(a.x, b.x), dy = __fsub_rn(a.y, b.y), dz = __fsub_rn(a.z, b.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Examines the centres spos[rg.x, rg.y) (at most the rest of the budget) for p's list.
__device__ __forceinline__ void scan_cell(float4 p, uint2 rg, const float4 *spos, uint32_t &examined, float (&bd)[kK],
                                          uint32_t (&bi)[kK]) {
    const uint32_t end = min(rg.y, rg.x + (kQueryBudget - min(examined, kQueryBudget)));
    examined += rg.y - rg.x;
    for (uint32_t q = rg.x; q < end; ++q) {
        const float4 o = __ldg(spos + q);
        const float d = dist2(p, o);
        uint32_t id = __float_as_uint(o.w);
        if (d > bd[kK - 1] || (d == bd[kK - 1] && id >= bi[kK - 1])) continue;
        float cd = d;
#pragma unroll
        for (int k = 0; k < kK; ++k) {  // insert, keeping (distance, index) order
            const bool less = cd < bd[k] || (cd == bd[k] && id < bi[k]);
            const float td = bd[k];
            const uint32_t ti = bi[k];
            bd[k] = less ? cd : td;
            bi[k] = less ? id : ti;
            cd = less ? td : cd;
            id = less ? ti : id;
        }
    }
}

// Ring search around point p for its kK nearest centres (lists in bd / bi, sorted).
__device__ __forceinline__ void ring_search(float4 p, const KnnGrid &G, const uint2 *ranges, const float4 *spos,
                                            float (&bd)[kK], uint32_t (&bi)[kK]) {
    const int c[3] = {cell_axis(p.x, G.lo[0], G.inv_h, G.dims[0]), cell_axis(p.y, G.lo[1], G.inv_h, G.dims[1]),
                      cell_axis(p.z, G.lo[2], G.inv_h, G.dims[2])};
    const float pc[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int k = 0; k < kK; ++k) { bd[k] = __int_as_float(0x7f800000); bi[k] = 0xffffffffu; }
    const int rmax = max(max(G.dims[0], G.dims[1]), G.dims[2]);
    // distance along axis k from p to cell index ci's slab, less the rounding slack; once 16
    // are held, a row or cell whose box is farther than the 16th is skipped unread
    auto gap = [&](int k, int ci) {
        const float a = G.lo[k] + (float)ci * G.h - G.slack - pc[k];
        const float b = pc[k] - (G.lo[k] + (float)(ci + 1) * G.h + G.slack);
        return fmaxf(fmaxf(a, b), 0.f);
    };
    float outg[3], og2 = 0.f;  // distance from p to the grid's box along each axis, less the slack
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        outg[k] = fmaxf(fmaxf(G.lo[k] - G.slack - pc[k], pc[k] - (G.lo[k] + (float)G.dims[k] * G.h + G.slack)), 0.f);
        og2 = fmaf(outg[k], outg[k], og2);
    }
    uint32_t examined = 0;
    for (int ring = 0; ring <= rmax && examined < kQueryBudget; ++ring) {
        const int z0 = max(c[2] - ring, 0), z1 = min(c[2] + ring, G.dims[2] - 1);
        const int y0 = max(c[1] - ring, 0), y1 = min(c[1] + ring, G.dims[1] - 1);
        const int x0 = max(c[0] - ring, 0), x1 = min(c[0] + ring, G.dims[0] - 1);
        auto visit = [&](int cx, int cy, int cz, float gyz) {
            const float gx = gap(0, cx);
            if (fmaf(gx, gx, gyz) > bd[kK - 1]) return;
            scan_cell(p, __ldg(ranges + (cx + G.dims[0] * (cy + G.dims[1] * cz))), spos, examined, bd, bi);
        };
        // the cells at Chebyshev distance `ring` from the query's cell
        for (int cz = z0; cz <= z1; ++cz) {
            const float gz = gap(2, cz);
            if (gz * gz > bd[kK - 1]) continue;
            for (int cy = y0; cy <= y1; ++cy) {
                const float gy = gap(1, cy);
                const float gyz = fmaf(gy, gy, gz * gz);
                if (gyz > bd[kK - 1]) continue;
                if (abs(cz - c[2]) < ring && abs(cy - c[1]) < ring) {  // only the two x faces are new
                    if (c[0] - ring >= 0) visit(c[0] - ring, cy, cz, gyz);
                    if (c[0] + ring < G.dims[0]) visit(c[0] + ring, cy, cz, gyz);
                } else {
                    for (int cx = x0; cx <= x1; ++cx) visit(cx, cy, cz, gyz);
                }
            }
        }
        // every unsearched point lies in the grid's box beyond one of the searched block's open
        // faces; b2 is the least squared distance from p to those regions (a query outside the
        // box adds its distance to the box on the other axes)
        float b2 = __int_as_float(0x7f800000);
        bool all = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float others = og2 - outg[k] * outg[k];
            if (c[k] - ring > 0) {
                const float g = fmaxf(pc[k] - (G.lo[k] + (float)(c[k] - ring) * G.h) - G.slack, 0.f);
                b2 = fminf(b2, fmaf(g, g, others));
                all = false;
            }
            if (c[k] + ring < G.dims[k] - 1) {
                const float g = fmaxf((G.lo[k] + (float)(c[k] + ring + 1) * G.h) - pc[k] - G.slack, 0.f);
                b2 = fminf(b2, fmaf(g, g, others));
                all = false;
            }
        }
        if (all) break;
        if (bi[kK - 1] != 0xffffffffu && bd[kK - 1] <= b2 * (1.f - 1.f / 1048576.f)) break;
    }
}

// Distance from p to the slab [lo + i w, lo + (i + 1) w] of one axis, less the slack.
__device__ __forceinline__ float slab_gap(float lo, float w, float slack, float p, int i) {
    return fmaxf(fmaxf(lo + (float)i * w - slack - p, p - (lo + (float)(i + 1) * w + slack)), 0.f);
}

// The same search over Chebyshev rings of 2 x 2 x 2-cell blocks, for queries anywhere in
// space (start points in front of a surface, rays past its edge): a block whose box lies
// farther than the 16th candidate, or that holds no centre, costs one test and at most one
// count read; the cells of the others are pruned and scanned as in ring_search.
__device__ __forceinline__ void block_search(float4 p, const KnnGrid G, const uint2 *ranges, const uint32_t *bcount,
                                             const float4 *spos, float (&bd)[kK], uint32_t (&bi)[kK]) {
    const int dx = G.dims[0], dy = G.dims[1], dz = G.dims[2];
    const int bx_n = block_dim(dx), by_n = block_dim(dy), bz_n = block_dim(dz);
    const int cbx = cell_axis(p.x, G.lo[0], G.inv_h, dx) >> 1, cby = cell_axis(p.y, G.lo[1], G.inv_h, dy) >> 1,
              cbz = cell_axis(p.z, G.lo[2], G.inv_h, dz) >> 1;
    const float h = G.h, H = G.h + G.h, sl = G.slack;
    const float lx = G.lo[0], ly = G.lo[1], lz = G.lo[2];
#pragma unroll
    for (int k = 0; k < kK; ++k) { bd[k] = __int_as_float(0x7f800000); bi[k] = 0xffffffffu; }
    // distance from p to the grid's box along each axis
    const float ox = fmaxf(fmaxf(lx - sl - p.x, p.x - (lx + (float)dx * h + sl)), 0.f);
    const float oy = fmaxf(fmaxf(ly - sl - p.y, p.y - (ly + (float)dy * h + sl)), 0.f);
    const float oz = fmaxf(fmaxf(lz - sl - p.z, p.z - (lz + (float)dz * h + sl)), 0.f);
    const int rmax = max(max(bx_n, by_n), bz_n);
    uint32_t examined = 0;
    for (int ring = 0; ring <= rmax && examined < kQueryBudget; ++ring) {
        const int z0 = max(cbz - ring, 0), z1 = min(cbz + ring, bz_n - 1);
        const int y0 = max(cby - ring, 0), y1 = min(cby + ring, by_n - 1);
        const int x0 = max(cbx - ring, 0), x1 = min(cbx + ring, bx_n - 1);
        auto visit = [&](int bx, int by, int bz, float gyz) {
            const float gx = slab_gap(lx, H, sl, p.x, bx);
            if (fmaf(gx, gx, gyz) > bd[kK - 1]) return;
            if (__ldg(bcount + (bx + bx_n * (by + by_n * bz))) == 0u) return;
            const int fz1 = min(2 * bz + 1, dz - 1), fy1 = min(2 * by + 1, dy - 1), fx1 = min(2 * bx + 1, dx - 1);
            for (int fz = 2 * bz; fz <= fz1; ++fz) {
                const float hz = slab_gap(lz, h, sl, p.z, fz);
                for (int fy = 2 * by; fy <= fy1; ++fy) {
                    const float hy = slab_gap(ly, h, sl, p.y, fy);
                    const float hyz = fmaf(hy, hy, hz * hz);
                    if (hyz > bd[kK - 1]) continue;
                    for (int fx = 2 * bx; fx <= fx1; ++fx) {
                        const float hx = slab_gap(lx, h, sl, p.x, fx);
                        if (fmaf(hx, hx, hyz) > bd[kK - 1]) continue;
                        scan_cell(p, __ldg(ranges + (fx + dx * (fy + dy * fz))), spos, examined, bd, bi);
                    }
                }
            }
        };
        for (int bz = z0; bz <= z1; ++bz) {
            const float gz = slab_gap(lz, H, sl, p.z, bz);
            if (gz * gz > bd[kK - 1]) continue;
            for (int by = y0; by <= y1; ++by) {
                const float gy = slab_gap(ly, H, sl, p.y, by);
                const float gyz = fmaf(gy, gy, gz * gz);
                if (gyz > bd[kK - 1]) continue;
                if (abs(bz - cbz) < ring && abs(by - cby) < ring) {  // only the two x faces are new
                    if (cbx - ring >= 0) visit(cbx - ring, by, bz, gyz);
                    if (cbx + ring < bx_n) visit(cbx + ring, by, bz, gyz);
                } else {
                    for (int bx = x0; bx <= x1; ++bx) visit(bx, by, bz, gyz);
                }
            }
        }
        // least distance to the grid's box beyond the searched blocks' open faces
        float b2 = __int_as_float(0x7f800000);
        bool all = true;
        auto face = [&](bool open, float g, float o1, float o2) {
            if (!open) return;
            g = fmaxf(g - sl, 0.f);
            b2 = fminf(b2, fmaf(g, g, fmaf(o1, o1, o2 * o2)));
            all = false;
        };
        face(cbx - ring > 0, p.x - (lx + (float)(cbx - ring) * H), oy, oz);
        face(cbx + ring < bx_n - 1, (lx + (float)(cbx + ring + 1) * H) - p.x, oy, oz);
        face(cby - ring > 0, p.y - (ly + (float)(cby - ring) * H), ox, oz);
        face(cby + ring < by_n - 1, (ly + (float)(cby + ring + 1) * H) - p.y, ox, oz);
        face(cbz - ring > 0, p.z - (lz + (float)(cbz - ring) * H), ox, oy);
        face(cbz + ring < bz_n - 1, (lz + (float)(cbz + ring + 1) * H) - p.z, ox, oy);
        if (all) break;
        if (bi[kK - 1] != 0xffffffffu && bd[kK - 1] <= b2 * (1.f - 1.f / 1048576.f)) break;
    }
}

__global__ void __launch_bounds__(128) k_knn_query(const float4 *spos, const uint2 *ranges, const KnnGrid *gp, int n,
                                                   int32_t *knn) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const float4 p = spos[r];
    float bd[kK];
    uint32_t bi[kK];
    ring_search(p, *gp, ranges, spos, bd, bi);
    int32_t *out = knn + (size_t)__float_as_uint(p.w) * kK;
#pragma unroll
    for (int k = 0; k < kK; ++k) out[k] = (int32_t)bi[k];
}

// Cell keys of query points (w = 0: no query, sorted after every cell).
__global__ void __launch_bounds__(256) k_knn_point_keys(const float4 *pts, int m, const KnnGrid *g, uint32_t none,
                                                        uint32_t *keys) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const float4 p = pts[r];
    const KnnGrid G = *g;
    keys[r] = p.w == 0.f ? none
                         : (uint32_t)(cell_axis(p.x, G.lo[0], G.inv_h, G.dims[0]) +
                                      G.dims[0] * (cell_axis(p.y, G.lo[1], G.inv_h, G.dims[1]) +
                                                   G.dims[1] * cell_axis(p.z, G.lo[2], G.inv_h, G.dims[2])));
}

// Queries at arbitrary points, taken in cell order (order[r]: the r-th query by cell), so a
// warp searches one neighbourhood; w = 0: no query, the list is all -1.
__global__ void __launch_bounds__(32) k_knn_points(const float4 *spos, const uint2 *ranges, const uint32_t *bcount,
                                                    const KnnGrid *gp, const float4 *pts, const uint32_t *order, int m,
                                                    int32_t *knn) {
    const int r0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (r0 >= m) return;
    const uint32_t r = __ldg(order + r0);
    const float4 p = pts[r];
    float bd[kK];
    uint32_t bi[kK];
    if (p.w != 0.f) {
        const KnnGrid G = *gp;
        block_search(p, G, ranges, bcount, spos, bd, bi);
    } else {
#pragma unroll
        for (int k = 0; k < kK; ++k) bi[k] = 0xffffffffu;
    }
    int4 *out = reinterpret_cast<int4 *>(knn + (size_t)r * kK);
#pragma unroll
    for (int k = 0; k < kK; k += 4)
        out[k / 4] = make_int4((int32_t)bi[k], (int32_t)bi[k + 1], (int32_t)bi[k + 2], (int32_t)bi[k + 3]);
}

// Cell sort of m query points, after the grid's own workspace.
struct KnnQueryLayout {
    uint64_t keys0, keys1, vals0, vals1, hist, partials, bytes;
    uint32_t nblocks;
    int bits;
};

KnnQueryLayout knn_query_layout(uint32_t cap_cells, int32_t m) {
    KnnQueryLayout Q;
    Q.bits = 1;
    while ((1ull << Q.bits) <= cap_cells) ++Q.bits;  // every cell index and the "no query" key fit
    Q.nblocks = ceil_div_u64(m > 0 ? (uint64_t)m : 1, kSortTile);
    uint64_t off = 0;
    Q.keys0 = off; off = al256(off + 4ull * m);
    Q.keys1 = off; off = al256(off + 4ull * m);
    Q.vals0 = off; off = al256(off + 4ull * m);
    Q.vals1 = off; off = al256(off + 4ull * m);
    Q.hist = off; off = al256(off + 4ull * 256 * Q.nblocks);
    Q.partials = off; off = al256(off + 4ull * (ceil_div_u64(256ull * Q.nblocks, kScanTile) + 1));
    Q.bytes = off;
    return Q;
}

template <class T>
T *at(void *base, uint64_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" size_t ges_knn_workspace_bytes(int32_t n) {
    if (n < GES_KNN_K || (uint64_t)n > (1ull << 26)) return 0;
    return knn_layout(n).bytes;
}

namespace ges {

// Grid, cell sort and cell-ordered centres of n splats in `workspace` (knn_layout(n).bytes).
static cudaError_t knn_build(int32_t n, const float4 *pos, void *workspace, const KnnLayout &L, cudaStream_t s) {
    uint32_t *bb = at<uint32_t>(workspace, L.bbox);
    KnnGrid *grid = at<KnnGrid>(workspace, L.grid);
    cudaError_t e = cudaMemsetAsync(bb, 0xff, 12, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bb + 3, 0, 12, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(at<void>(workspace, L.ranges), 0, 8ull * L.cap_cells, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(at<void>(workspace, L.bcount), 0, 4ull * L.cap_cells, s);
    if (e != cudaSuccess) return e;
    k_knn_bbox<<<min(ceil_div_u64(n, 256), 1024u), 256, 0, s>>>(pos, n, bb);
    k_knn_grid<<<1, 1, 0, s>>>(bb, L.cap_cells, grid);
    uint32_t *keys[2] = {at<uint32_t>(workspace, L.keys0), at<uint32_t>(workspace, L.keys1)};
    uint32_t *vals[2] = {at<uint32_t>(workspace, L.vals0), at<uint32_t>(workspace, L.vals1)};
    k_knn_keys<<<ceil_div_u64(n, 256), 256, 0, s>>>(pos, n, grid, keys[0], at<uint32_t>(workspace, L.bcount));
    e = radix_sort(keys, vals, true, nullptr, (uint32_t)n, L.bits, at<uint32_t>(workspace, L.hist),
                   at<uint32_t>(workspace, L.partials), s);
    if (e != cudaSuccess) return e;
    const int res = ((L.bits + 7) / 8) & 1;
    k_knn_ranges<<<ceil_div_u64(n, 256), 256, 0, s>>>(keys[res], vals[res], pos, n, at<uint2>(workspace, L.ranges),
                                                     at<float4>(workspace, L.spos));
    return cudaGetLastError();
}

// Workspace of knn_points_run: the grid of n centres, then the cell sort of m queries.
size_t knn_points_workspace(int32_t n, int32_t m) {
    const KnnLayout L = knn_layout(n);
    return L.bytes + knn_query_layout(L.cap_cells, m).bytes;
}

// The 16 nearest centres of m points (pts[i].w = 0: none, list -1) into knn [m][16]
// (16-byte aligned); workspace: knn_points_workspace(n, m) bytes, 256-byte aligned.
cudaError_t knn_points_run(int32_t n, const float4 *pos, int32_t m, const float4 *pts, void *workspace,
                           int32_t *knn, cudaStream_t s) {
    const KnnLayout L = knn_layout(n);
    cudaError_t e = knn_build(n, pos, workspace, L, s);
    if (e != cudaSuccess || m <= 0) return e;
    const KnnQueryLayout Q = knn_query_layout(L.cap_cells, m);
    void *qws = static_cast<char *>(workspace) + L.bytes;
    uint32_t *keys[2] = {at<uint32_t>(qws, Q.keys0), at<uint32_t>(qws, Q.keys1)};
    uint32_t *vals[2] = {at<uint32_t>(qws, Q.vals0), at<uint32_t>(qws, Q.vals1)};
    k_knn_point_keys<<<ceil_div_u64(m, 256), 256, 0, s>>>(pts, m, at<KnnGrid>(workspace, L.grid),
                                                          (uint32_t)((1ull << Q.bits) - 1), keys[0]);
    e = radix_sort(keys, vals, true, nullptr, (uint32_t)m, Q.bits, at<uint32_t>(qws, Q.hist),
                   at<uint32_t>(qws, Q.partials), s);
    if (e != cudaSuccess) return e;
    const int res = ((Q.bits + 7) / 8) & 1;
    // one warp per CTA: query walks differ widely in length, and a CTA of several warps would hold
    // its slot until its longest walk ended
    k_knn_points<<<ceil_div_u64(m, 32), 32, 0, s>>>(at<float4>(workspace, L.spos), at<uint2>(workspace, L.ranges),
                                                     at<uint32_t>(workspace, L.bcount), at<KnnGrid>(workspace, L.grid),
                                                     pts, vals[res], m, knn);
    return cudaGetLastError();
}

}  // namespace ges

extern "C" ges_status ges_knn(int32_t n, const float *pos_op, void *workspace, size_t workspace_bytes, int32_t *knn,
                              void *stream) {
    GES_RANGE();
    if (n < GES_KNN_K || (uint64_t)n > (1ull << 26) || !pos_op || !workspace || !knn) return GES_ERR_INVALID_ARG;
    if (((uintptr_t)pos_op & 15u) || ((uintptr_t)workspace & 255u) || ((uintptr_t)knn & 3u))
        return GES_ERR_INVALID_ARG;
    const KnnLayout L = knn_layout(n);
    if (workspace_bytes < L.bytes) return GES_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const float4 *pos = reinterpret_cast<const float4 *>(pos_op);
    if (knn_build(n, pos, workspace, L, s) != cudaSuccess) return GES_ERR_CUDA;
    k_knn_query<<<ceil_div_u64(n, 128), 128, 0, s>>>(at<float4>(workspace, L.spos), at<uint2>(workspace, L.ranges),
                                                    at<KnnGrid>(workspace, L.grid), n, knn);
    return cudaGetLastError() == cudaSuccess ? GES_OK : GES_ERR_CUDA;
}

extern "C" size_t ges_knn_points_workspace_bytes(int32_t n, int32_t m) {
    if (n < GES_KNN_K || (uint64_t)n > (1ull << 26) || m < 1 || (uint64_t)m > (1ull << 28)) return 0;
    return knn_points_workspace(n, m);
}

extern "C" ges_status ges_knn_points(int32_t n, const float *pos_op, int32_t m, const float *points,
                                     void *workspace, size_t workspace_bytes, int32_t *knn, void *stream) {
    GES_RANGE();
    if (n < GES_KNN_K || (uint64_t)n > (1ull << 26) || m < 1 || (uint64_t)m > (1ull << 28)) return GES_ERR_INVALID_ARG;
    if (!pos_op || !points || !workspace || !knn) return GES_ERR_INVALID_ARG;
    if (((uintptr_t)pos_op & 15u) || ((uintptr_t)points & 15u) || ((uintptr_t)workspace & 255u) ||
        ((uintptr_t)knn & 15u))
        return GES_ERR_INVALID_ARG;
    if (workspace_bytes < knn_points_workspace(n, m)) return GES_ERR_INVALID_ARG;
    return knn_points_run(n, reinterpret_cast<const float4 *>(pos_op), m, reinterpret_cast<const float4 *>(points),
                          workspace, knn, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? GES_OK
               : GES_ERR_CUDA;
}
