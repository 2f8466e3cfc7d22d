// S5 binning: stable LSD radix sort (reduce-then-scan, 8-bit digits), exclusive
// scan, instance emission in depth order, tile ranges and the longest-first
// tile queue. Instance counts are read from device memory, so the whole chain
// runs without a host round trip and can be captured in a CUDA graph with
// capacity-sized grids (CTAs past the live count exit at once).
#include "ges_internal.cuh"
#include "tile_tests.cuh"

namespace ges {

// ------------------------------------------------------------------ scan
// Exclusive scan of n uint32 in three launches: tile sums, one-CTA scan of the
// tile sums, tile scans offset by the scanned sums. In place is allowed.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive block scan of one value per thread (blockDim.x multiple of 32, <= 1024).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t incl = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < nw) s_warp[lane] = wi - w;
        if (lane == 31) s_warp[32] = wi;
    }
    __syncthreads();
    uint32_t r = incl - v + s_warp[warp];
    total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t *in, uint32_t n, uint32_t *partials) {
    __shared__ uint32_t s_warp[33];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint32_t sum = 0;
#pragma unroll 4
    for (int k = 0; k < kScanTile / 256; ++k) {
        uint64_t idx = base + (uint64_t)k * 256 + threadIdx.x;
        if (idx < n) sum += in[idx];
    }
    uint32_t tot;
    block_excl_scan(sum, s_warp, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// One CTA of 1024 threads scans up to kScanMaxPartials tile sums; writes the grand total.
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *partials, uint32_t np, uint32_t *total) {
    __shared__ uint32_t s_warp[33];
    constexpr int PER = kScanMaxPartials / 1024;
    uint32_t v[PER];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        uint32_t idx = threadIdx.x * PER + k;
        v[k] = idx < np ? partials[idx] : 0u;
        s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_excl_scan(s, s_warp, tot);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        uint32_t idx = threadIdx.x * PER + k;
        if (idx < np) partials[idx] = run;
        run += v[k];
    }
    if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void __launch_bounds__(256) k_scan_down(const uint32_t *in, uint32_t *out, uint32_t n,
                                                  const uint32_t *partials) {
    __shared__ uint32_t s_data[kScanTile + kScanTile / 32];
    __shared__ uint32_t s_warp[33];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    constexpr int PER = kScanTile / 256;  // 16
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        uint32_t li = k * 256 + threadIdx.x;
        uint64_t idx = base + li;
        s_data[li + (li >> 5)] = idx < n ? in[idx] : 0u;
    }
    __syncthreads();
    uint32_t v[PER];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        uint32_t li = threadIdx.x * PER + k;
        v[k] = s_data[li + (li >> 5)];
        s += v[k];
    }
    uint32_t tot;
    uint32_t run = block_excl_scan(s, s_warp, tot) + partials[blockIdx.x];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        uint32_t li = threadIdx.x * PER + k;
        s_data[li + (li >> 5)] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        uint32_t li = k * 256 + threadIdx.x;
        uint64_t idx = base + li;
        if (idx < n) out[idx] = s_data[li + (li >> 5)];
    }
}

cudaError_t exclusive_scan(const uint32_t *in, uint32_t *out, uint32_t n, uint32_t *partials, uint32_t *total,
                           cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t nb = ceil_div_u64(n, kScanTile);
    if (nb > (uint32_t)kScanMaxPartials) return cudaErrorInvalidValue;
    k_scan_reduce<<<nb, 256, 0, s>>>(in, n, partials);
    k_scan_partials<<<1, 1024, 0, s>>>(partials, nb, total);
    k_scan_down<<<nb, 256, 0, s>>>(in, out, n, partials);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ radix sort
// Count source: n_dev (device, clamped to cap) if given, else n_host.
__device__ __forceinline__ uint32_t live_count(const uint32_t *n_dev, uint32_t n_host) {
    return n_dev ? *n_dev : n_host;
}

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *keys, const uint32_t *n_dev,
                                                            uint32_t n_host, int shift, uint32_t nblocks,
                                                            uint32_t *hist) {
    __shared__ uint32_t s_h[kSortThreads / 32][256];
    const int warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < (kSortThreads / 32) * 256; k += kSortThreads) (&s_h[0][0])[k] = 0u;
    __syncthreads();
    const uint32_t n = live_count(n_dev, n_host);
    const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
    if (base < n) {
        uint32_t kk[kSortItems];
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint64_t idx = base + (uint64_t)k * kSortThreads + threadIdx.x;
            kk[k] = idx < n ? __ldg(keys + idx) : 0xffffffffu;
        }
#pragma unroll
        for (int k = 0; k < kSortItems; ++k) {
            const uint64_t idx = base + (uint64_t)k * kSortThreads + threadIdx.x;
            if (idx < n) atomicAdd(&s_h[warp][(kk[k] >> shift) & 0xffu], 1u);
        }
    }
    __syncthreads();
    const int d = threadIdx.x;  // kSortThreads == 256 digits
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) c += s_h[w][d];
    hist[(uint64_t)d * nblocks + blockIdx.x] = c;
}

// Stable scatter: each warp ranks a contiguous 512-key chunk in rounds of 32 with
// digit ballots, keeping a per-warp running count per digit; warps are then ordered by
// an exclusive prefix per digit. The CTA's 4096 pairs are first reordered by digit
// in shared memory, then written out in digit runs (coalesced) at the offsets of
// the scanned digit-major histogram.
__global__ void __launch_bounds__(kSortThreads, 3) k_radix_scatter(const uint32_t *keys_in, const uint32_t *vals_in,
                                                               uint32_t *keys_out, uint32_t *vals_out,
                                                               const uint32_t *n_dev, uint32_t n_host, int shift,
                                                               uint32_t nblocks, const uint32_t *hist_scanned) {
    constexpr int NW = kSortThreads / 32;
    __shared__ uint32_t s_cnt[NW][256];
    __shared__ uint32_t s_dstart[256], s_gstart[256];
    __shared__ uint32_t s_warp[33];
    __shared__ uint32_t s_keys[kSortTile], s_vals[kSortTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < NW * 256; k += kSortThreads) (&s_cnt[0][0])[k] = 0u;
    __syncthreads();
    const uint32_t n = live_count(n_dev, n_host);
    const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
    if (base >= n) return;  // uniform for the CTA
    const uint32_t nvalid = (uint32_t)min((uint64_t)kSortTile, (uint64_t)n - base);
    const uint64_t wbase = base + (uint64_t)warp * (kSortItems * 32);
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
    // all loads first, so that the 16 rounds' reads are in flight together
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
        const bool valid = idx < n;
        key[r] = valid ? __ldg(keys_in + idx) : 0u;
        val[r] = valid ? (vals_in ? __ldg(vals_in + idx) : (uint32_t)idx) : 0u;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint64_t idx = wbase + (uint64_t)r * 32 + lane;
        const bool valid = idx < n;
        const uint32_t d = (key[r] >> shift) & 0xffu;
        // lanes holding the same digit (invalid lanes carry 0x100): one ballot per digit
        // bit, which issues faster than match.any on spread-out digits
        const uint32_t dd = valid ? d : 0x100u;
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (dd >> b) & 1u);
            peers &= ((dd >> b) & 1u) ? bal : ~bal;
        }
        uint32_t before = 0;
        if (valid) before = s_cnt[warp][d];
        __syncwarp();
        if (valid && (peers & lt_mask) == 0) s_cnt[warp][d] = before + __popc(peers);
        __syncwarp();
        rank[r] = valid ? before + __popc(peers & lt_mask) : 0xffffffffu;
    }
    __syncthreads();
    {
        // digit d = thread: block count, block-local start (exclusive scan over digits),
        // per-warp offsets inside the digit, and the digit's global start for this CTA
        const int d = threadIdx.x;
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) c += s_cnt[w][d];
        uint32_t tot;
        const uint32_t start = block_excl_scan(c, s_warp, tot);
        s_dstart[d] = start;
        s_gstart[d] = hist_scanned[(uint64_t)d * nblocks + blockIdx.x];
        uint32_t run = start;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t t = s_cnt[w][d];
            s_cnt[w][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        if (rank[r] == 0xffffffffu) continue;
        const uint32_t d = (key[r] >> shift) & 0xffu;
        const uint32_t lpos = s_cnt[warp][d] + rank[r];
        s_keys[lpos] = key[r];
        s_vals[lpos] = val[r];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nvalid; i += kSortThreads) {
        const uint32_t k = s_keys[i];
        const uint32_t d = (k >> shift) & 0xffu;
        const uint32_t pos = s_gstart[d] + (i - s_dstart[d]);
        if (keys_out) keys_out[pos] = k;
        vals_out[pos] = s_vals[i];
    }
}

// Sorts (keys, vals) on bits [0, bits) with ceil(bits/8) passes, ping-ponging
// between buffer 0 and 1; the result lands in buffer (passes % 2). vals[0] may be
// NULL for "value = index". Keys are always written (tile ranges need them).
cudaError_t radix_sort(uint32_t *keys[2], uint32_t *vals[2], bool iota_vals, const uint32_t *n_dev,
                       uint32_t n_host_max, int bits, uint32_t *hist, uint32_t *partials, cudaStream_t s) {
    const uint32_t nblocks = ceil_div_u64(n_host_max > 0 ? n_host_max : 1, kSortTile);
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int in = p & 1, out = in ^ 1;
        const int shift = 8 * p;
        k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(keys[in], n_dev, n_host_max, shift, nblocks, hist);
        cudaError_t e = exclusive_scan(hist, hist, 256u * nblocks, partials, nullptr, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(keys[in], (p == 0 && iota_vals) ? nullptr : vals[in],
                                                        keys[out], vals[out], n_dev, n_host_max, shift, nblocks,
                                                        hist);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ emission

// Depth order -> tiles touched per rank (scanned next into emission offsets), and a
// rank-ordered copy of what emission needs, so that k_emit streams instead of
// gathering the binning records a second time. rinfo per rank: entry, hit mask,
// global key of the tile box's first tile, and (box width in tiles | view tiles
// per row << 6); box width 0 marks a box of more than 32 tiles (no mask).
__global__ void __launch_bounds__(128) k_gather_counts(const uint32_t *sorted_e, const uint4 *binrec,
                                                      uint32_t *counts, uint4 *rinfo, uint32_t n_entries, int n,
                                                      ViewSet V) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_entries) return;
    const uint32_t e = __ldg(sorted_e + r);
    // both halves of the 32-byte record in one round trip
    const uint4 b0 = __ldg(binrec + 2 * (size_t)e), b1 = __ldg(binrec + 2 * (size_t)e + 1);
    const uint32_t tiles = b0.z;
    counts[r] = tiles;
    if (tiles) {
        const int v = (int)(e / (uint32_t)n);
        const int tx0 = (int)(b1.y & 0xffffu), ty0 = (int)(b1.y >> 16);
        const int rw = (int)(b1.z & 0xffffu), rh = (int)(b1.z >> 16);
        const int tiles_x = V.tiles_x[v];
        const uint32_t origin = (uint32_t)V.tile_base[v] + (uint32_t)(ty0 * tiles_x + tx0);
        const uint32_t shape = (rw * rh <= 32 ? (uint32_t)rw : 0u) | ((uint32_t)tiles_x << 6);
        rinfo[r] = make_uint4(e, b1.x, origin, shape);
    }
}

// Position of the k-th (0-based) set bit of m; m has more than k set bits.
__device__ __forceinline__ uint32_t select_bit(uint32_t m, uint32_t k) {
    uint32_t pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const uint32_t lo = m & ((1u << s) - 1u);
        const uint32_t c = (uint32_t)__popc(lo);
        if (k >= c) { k -= c; m >>= s; pos += s; } else { m = lo; }
    }
    return pos;
}

// Emission. Ranks r..r+31 of a warp own the contiguous instance range
// [offsets[r], offsets[r+32]); the warp expands their hit masks together, 32
// instances per round: instance j goes to the rank whose prefix interval holds j
// (binary search over the warp's inclusive prefix) and to that rank's j-th set
// mask bit. Writes are coalesced. Boxes of more than 32 tiles (no mask) are
// expanded afterwards by their own lane with the tile test.
__global__ void __launch_bounds__(128) k_emit(EmitArgs a) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned long long total = *a.total;
    if (total >= 0xffffffffull) {  // uint32 offsets would wrap
        if (r == 0) set_error(a.err, kErrCapacity);
        return;
    }
    if (blockIdx.x * blockDim.x + (threadIdx.x & ~31u) >= a.n_entries) return;  // whole warp past the end
    const bool live = r < a.n_entries;
    uint32_t off = 0, tiles = 0;
    if (live) {
        off = a.offsets[r];
        const uint32_t next = (r + 1 < a.n_entries) ? a.offsets[r + 1] : (uint32_t)total;
        tiles = next > off ? next - off : 0u;
    }
    if (tiles && (uint64_t)off + tiles > a.cap) set_error(a.err, kErrCapacity);
    uint4 info = make_uint4(0u, 0u, 0u, 0u);
    if (tiles) info = a.rinfo[r];
    const uint32_t rw = info.w & 63u;
    const uint32_t cnt = rw ? tiles : 0u;  // instances expanded cooperatively
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    const uint32_t wtotal = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - cnt;
    const uint32_t mdiv = rw ? (65536u + rw - 1u) / rw : 0u;  // bit / rw == (bit * mdiv) >> 16 for bit < 32
    const uint32_t base = off - excl;                          // instance j of the warp lands at base + j
    for (uint32_t j0 = 0; j0 < wtotal; j0 += 32) {
        const uint32_t j = j0 + (uint32_t)lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t p = __shfl_sync(0xffffffffu, incl, owner + step - 1);
            if (p <= j) owner += step;
        }
        const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, owner);
        const uint32_t o_base = __shfl_sync(0xffffffffu, base, owner);
        const uint32_t o_mask = __shfl_sync(0xffffffffu, info.y, owner);
        const uint32_t o_org = __shfl_sync(0xffffffffu, info.z, owner);
        const uint32_t o_shape = __shfl_sync(0xffffffffu, info.w, owner);
        const uint32_t o_mdiv = __shfl_sync(0xffffffffu, mdiv, owner);
        const uint32_t o_e = __shfl_sync(0xffffffffu, info.x, owner);
        if (j < wtotal) {
            const uint32_t bit = select_bit(o_mask, j - o_excl);
            const uint32_t row = (bit * o_mdiv) >> 16;
            const uint32_t col = bit - row * (o_shape & 63u);
            const uint64_t pos = (uint64_t)o_base + j;
            if (pos < a.cap) {
                a.ikey[pos] = o_org + row * (o_shape >> 6) + col;
                a.ival[pos] = o_e;
            }
        }
    }
    // boxes of more than 32 tiles: the tile tests spread over the warp, each hit
    // written at its entry's offset plus the number of earlier hits of that entry
    // (row-major order, as a per-entry loop over the box would write them)
    const bool big = tiles && !rw;
    if (!__any_sync(0xffffffffu, big)) return;
    const int tw = a.V.tile_w, th = a.V.tile_h;
    const int lw = __ffs(tw) - 1, lh = __ffs(th) - 1;  // tile sides are powers of two
    TileJob J = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, 0u, 0u};
    uint32_t tbase = 0;
    int tiles_x = 0;
    if (big) {
        const uint32_t e = info.x;
        const int v = (int)(e / (uint32_t)a.n);
        tbase = (uint32_t)a.V.tile_base[v];
        tiles_x = a.V.tiles_x[v];
        const uint4 br = a.binrec[2 * (size_t)e];
        const float4 r0 = a.rec[4 * (size_t)e], r1 = a.rec[4 * (size_t)e + 1];
        int x0, x1, y0, y1;
        pixel_box(r0.x, r0.y, __uint_as_float(br.x), __uint_as_float(br.y), a.V.width[v], a.V.height[v], x0, x1,
                  y0, y1);
        if (x0 <= x1 && y0 <= y1)
            J = TileJob{r0.x, r0.y, r0.z, r0.w, r1.x, __frcp_rn(r0.z), __frcp_rn(r1.x), __fmul_rn(r1.y, kSupportMargin),
                        (uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16),
                        (uint32_t)((x1 >> lw) - (x0 >> lw) + 1) * (uint32_t)((y1 >> lh) - (y0 >> lh) + 1)};
    }
    uint32_t written = 0;  // hits of this lane's entry written so far
    __shared__ uint4 s_jobs[4][kJobWords * 32];  // 128 threads: 4 warps
    warp_tile_rounds(J, lane, lw, lh, tw, th, s_jobs[threadIdx.x >> 5],
                     [&](uint32_t hits, uint32_t lo, uint32_t len, uint32_t, int tx, int ty, uint32_t owner,
                         bool hit) {
                         const uint32_t o_off = __shfl_sync(0xffffffffu, off, owner);
                         const uint32_t o_written = __shfl_sync(0xffffffffu, written, owner);
                         const uint32_t o_tbase = __shfl_sync(0xffffffffu, tbase, owner);
                         const int o_tiles_x = __shfl_sync(0xffffffffu, tiles_x, owner);
                         const uint32_t o_e = __shfl_sync(0xffffffffu, info.x, owner);
                         const uint32_t same = __match_any_sync(0xffffffffu, owner);
                         if (hit) {
                             const uint64_t pos = (uint64_t)o_off + o_written +
                                                  (uint32_t)__popc(hits & same & ((1u << lane) - 1u));
                             if (pos < a.cap) {
                                 a.ikey[pos] = o_tbase + (uint32_t)(ty * o_tiles_x + tx);
                                 a.ival[pos] = o_e;
                             }
                         }
                         if (len)
                             written += (uint32_t)__popc((hits >> lo) &
                                                         (len == 32u ? 0xffffffffu : ((1u << len) - 1u)));
                     });
}

// n_inst = min(total, cap); 0 when the total does not fit the uint32 offsets
// (k_emit then writes nothing and records the capacity error).
__global__ void k_set_count(const unsigned long long *total, uint64_t cap, uint32_t *n_inst) {
    unsigned long long t = *total;
    *n_inst = t >= 0xffffffffull ? 0u : (uint32_t)(t < cap ? t : cap);
}

// Tile ranges from the sorted instance keys: thread q looks at keys 4q .. 4q+3 (one 16-byte load;
// the key buffer is capacity-sized and 256-byte aligned inside `bins`, so the load stays inside the
// allocation; keys at n and beyond are never used) and at their neighbours 4q - 1 and 4q + 4.
__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t *keys, const uint32_t *n_dev, uint2 *ranges,
                                                    uint32_t n_tiles) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t n = *n_dev;
    const uint32_t i0 = 4 * q;
    if (i0 >= n) return;
    const uint4 v = reinterpret_cast<const uint4 *>(keys)[q];
    const uint32_t k[6] = {i0 > 0 ? keys[i0 - 1] : 0u, v.x, v.y, v.z, v.w, i0 + 4 < n ? keys[i0 + 4] : 0u};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t i = i0 + (uint32_t)j;
        if (i >= n) break;
        const uint32_t kk = k[j + 1];
        if (kk >= n_tiles) continue;
        if (i == 0 || k[j] != kk) ranges[kk].x = i;
        if (i == n - 1 || k[j + 2] != kk) ranges[kk].y = i + 1;
    }
}

// Longest-first tile queue: tiles are bucketed by list length on a log2 scale
// (4 buckets per octave, longest first) with a one-CTA counting sort. Approximate
// LPT order is enough for scheduling; the results do not depend on it.
__global__ void __launch_bounds__(1024) k_lpt_queue(const uint2 *ranges, uint32_t n_tiles, uint32_t *queue) {
    constexpr int NB = 128;
    __shared__ uint32_t s_cnt[NB], s_off[NB];
    if (threadIdx.x < NB) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    auto bucket = [](uint32_t len) -> int {
        if (len == 0) return NB - 1;
        const float l = 4.f * log2f((float)len + 1.f);
        int b = (NB - 2) - (int)l;
        return b < 0 ? 0 : b;
    };
    for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        atomicAdd(&s_cnt[bucket(r.y - r.x)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = 0; b < NB; ++b) { s_off[b] = run; run += s_cnt[b]; }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t pos = atomicAdd(&s_off[bucket(r.y - r.x)], 1u);
        queue[pos] = t;
    }
}


__global__ void __launch_bounds__(256) k_depth_keys(const uint4 *binrec, uint32_t *keys, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) keys[i] = binrec[2 * (size_t)i].w;
}

cudaError_t launch_bin(const BinArgs &a, cudaStream_t s) {
    cudaError_t e;
    const uint32_t nE = a.n_entries;
    if (nE == 0) {  // no splats: every tile is empty
        e = cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * (size_t)a.V.n_tiles, s);
        if (e != cudaSuccess) return e;
        if (a.build_queue) k_lpt_queue<<<1, 1024, 0, s>>>(a.ranges, (uint32_t)a.V.n_tiles, a.queue);
        return cudaGetLastError();
    }
    // 1. depth sort of all entries; key = z32 bits (culled: 0xffffffff), value = entry
    k_depth_keys<<<ceil_div_u64(nE, 256), 256, 0, s>>>(a.binrec, a.dkey[0], nE);
    uint32_t *dk[2] = {a.dkey[0], a.dkey[1]}, *dv[2] = {a.dval[0], a.dval[1]};
    e = radix_sort(dk, dv, true, nullptr, nE, 32, a.hist, a.partials, s);
    if (e != cudaSuccess) return e;
    const uint32_t *sorted_e = dv[0];  // 4 passes: result back in buffer 0
    // 2. tiles touched in depth order -> exclusive scan -> emission offsets
    k_gather_counts<<<ceil_div_u64(nE, 128), 128, 0, s>>>(sorted_e, a.binrec, a.rcount, a.rinfo, nE, a.n, a.V);
    e = exclusive_scan(a.rcount, a.rcount, nE, a.partials, nullptr, s);
    if (e != cudaSuccess) return e;
    k_set_count<<<1, 1, 0, s>>>(a.total, a.cap, a.header);
    // 3. emit (tile, entry) instances in depth order
    EmitArgs ea;
    ea.n_entries = nE; ea.n = a.n; ea.rinfo = a.rinfo; ea.offsets = a.rcount; ea.rec = a.rec;
    ea.binrec = a.binrec; ea.total = a.total; ea.ikey = a.ikey[0]; ea.ival = a.ival[0]; ea.cap = a.cap;
    ea.err = a.err; ea.V = a.V;
    k_emit<<<ceil_div_u64(nE, 128), 128, 0, s>>>(ea);
    // 4. stable sort by global tile id keeps the depth order inside each tile
    uint32_t *ik[2] = {a.ikey[0], a.ikey[1]}, *iv[2] = {a.ival[0], a.ival[1]};
    const uint32_t cap32 = (uint32_t)a.cap;
    if (a.tile_bits > 0 && a.cap > 0) {
        e = radix_sort(ik, iv, false, a.header, cap32, a.tile_bits, a.hist, a.partials, s);
        if (e != cudaSuccess) return e;
    }
    const int res = ((a.tile_bits + 7) / 8) & 1;
    // 5. tile ranges
    e = cudaMemsetAsync(a.ranges, 0, sizeof(uint2) * (size_t)a.V.n_tiles, s);
    if (e != cudaSuccess) return e;
    if (a.cap > 0) k_tile_ranges<<<ceil_div_u64(ceil_div_u64(a.cap, 4), 256), 256, 0, s>>>(ik[res], a.header, a.ranges, (uint32_t)a.V.n_tiles);
    // 6. longest-first queue for the persistent render
    if (a.build_queue) k_lpt_queue<<<1, 1024, 0, s>>>(a.ranges, (uint32_t)a.V.n_tiles, a.queue);
    return cudaGetLastError();
}

}  // namespace ges
