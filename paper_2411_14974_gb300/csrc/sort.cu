// Binning and sorting for the convex tile rasterizer (Sec. 3.2: convexes are binned into tiles
// and drawn in order of increasing camera distance to their centres).
//
//   1. records sorted by depth key (binary32 bits of the distance, stable, so equal depths keep
//      increasing record index = convex index within a view), on the low key bits in which the
//      drawn records' keys differ only (they share the others; undrawn records emit no pairs);
//   2. with several views, a stable pass by view groups the depth-ordered records view by view;
//   3. exclusive scan of the per-record tile counts in that order;
//   4. each record emits (view << b | tile index within its view, record index) pairs, tiles in
//      row-major order, with the tile's 8-bit block mask above the view bits when it fits;
//   5. stable radix sort of the pairs on the b tile bits only: every (view, tile) group ends up
//      contiguous and in (depth, index) order, as a single sort on (view, tile, depth, index)
//      would leave it, with no sort passes spent on the view bits;
//   6. [start, end) range of every (view, tile) group in the sorted pair list.
//
// The radix sort is a three-kernel LSD sort (digit histogram per tile of 4096 keys, scan of the
// digit-major histogram, stable scatter).  Ranks inside a block come from warp-level key matching
// (__match_any_sync) over warp-striped runs of keys, so the scatter is stable.
#include <utility>

#include "cs_common.cuh"
#include "cs_spec_math.cuh"

namespace cs {
namespace {

#if CS_CHECKED
__device__ unsigned int g_status_sort;  // bits of the failed index tests of this file's kernels
__device__ __forceinline__ bool checked(bool ok, unsigned bit) {
    if (!ok) atomicOr(&g_status_sort, bit);
    return ok;
}
#else
__device__ __forceinline__ bool checked(bool ok, unsigned) { return true; }
#endif


constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int SPINE_THREADS = 1024;
constexpr int SCAN_INLINE_BLOCKS = 1024;  // up to this many blocks, no spine kernel

constexpr int RADIX_THREADS = 256;
constexpr int RADIX_WARPS = RADIX_THREADS / 32;
constexpr int RADIX_ITEMS = 16;
constexpr int RADIX_TILE = RADIX_THREADS * RADIX_ITEMS;  // 4096 keys per block
constexpr int RADIX_MAX_BITS = 8;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Kernels of the sort chain may be launched as programmatic dependents of the chain kernel before
// them: each waits here for that grid to complete (its results, and by the same wait in every
// chain kernel those of all earlier ones, are then visible), and at once lets its own dependent
// be scheduled, so that launches overlap the tail of the previous kernel.
__device__ __forceinline__ void chain_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- scan -----------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long v, unsigned long long *sh,
                                                                   unsigned long long &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (w == 0) {
        unsigned long long s = lane < nw ? sh[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    const unsigned long long warp_prefix = w > 0 ? sh[w - 1] : 0ull;
    total = sh[nw - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__device__ __forceinline__ uint32_t scan_load(const uint32_t *in, const uint32_t *gather, int64_t i, int64_t n) {
    if (i >= n) return 0u;
    return gather ? in[gather[i]] : in[i];
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t *__restrict__ in,
                                                              const uint32_t *__restrict__ gather, int64_t n,
                                                              unsigned long long *__restrict__ partial) {
    chain_enter();
    __shared__ unsigned long long sh[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) s += scan_load(in, gather, base + j * SCAN_THREADS + threadIdx.x, n);
    unsigned long long total;
    block_exclusive_scan(s, sh, total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SPINE_THREADS) k_scan_spine(unsigned long long *__restrict__ partial, int64_t nb,
                                                              unsigned long long *__restrict__ total_out) {
    chain_enter();
    __shared__ unsigned long long sh[32];
    unsigned long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SPINE_THREADS) {
        const int64_t i = b0 + threadIdx.x;
        const unsigned long long v = i < nb ? partial[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_scan(v, sh, tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

// INLINE: partial holds the blocks' plain sums and every block adds up those in front of it (no
// spine kernel; used up to SCAN_INLINE_BLOCKS blocks), the last block writing the total
template <bool INLINE>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const uint32_t *__restrict__ in,
                                                            const uint32_t *__restrict__ gather, int64_t n,
                                                            const unsigned long long *__restrict__ partial,
                                                            uint32_t *__restrict__ out,
                                                            unsigned long long *__restrict__ total_out) {
    chain_enter();
    __shared__ unsigned long long sh[32];
    unsigned long long prefix;
    if (INLINE) {
        unsigned long long s = 0, tot;
        for (int64_t b = threadIdx.x; b < (int64_t)blockIdx.x; b += SCAN_THREADS) s += partial[b];
        (void)block_exclusive_scan(s, sh, tot);
        prefix = tot;
    } else {
        prefix = partial[blockIdx.x];
    }
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;  // blocked
    uint32_t v[SCAN_ITEMS];
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = scan_load(in, gather, base + j, n);
        s += v[j];
    }
    unsigned long long tot;
    unsigned long long run = block_exclusive_scan(s, sh, tot) + prefix;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (base + j < n) out[base + j] = (uint32_t)run;
        run += v[j];
    }
    if (INLINE && total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = prefix + tot;
}

// ---- radix sort -----------------------------------------------------------------------------
// key_sub is subtracted from every key read (the first pass of a rebased sort; 0 otherwise)
__global__ void __launch_bounds__(RADIX_THREADS) k_radix_upsweep(const uint32_t *__restrict__ keys, int64_t n,
                                                                 int shift, int nbits, uint32_t key_sub,
                                                                 uint32_t *__restrict__ hist, int64_t nblocks) {
    chain_enter();
    __shared__ uint32_t cnt[RADIX_WARPS][1 << RADIX_MAX_BITS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nbins = 1u << nbits, mask = nbins - 1;
    for (int i = threadIdx.x; i < RADIX_WARPS * (1 << RADIX_MAX_BITS); i += RADIX_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    // counts only (no ranks): each thread takes RADIX_ITEMS consecutive keys (16-byte loads) and
    // adds every run of equal digits with one shared atomic into its warp's histogram
    (void)lane;
    const int64_t base = (int64_t)blockIdx.x * RADIX_TILE + (int64_t)threadIdx.x * RADIX_ITEMS;
    uint32_t k[RADIX_ITEMS];
    int nk = 0;
    if (base + RADIX_ITEMS <= n && (reinterpret_cast<uintptr_t>(keys) & 15) == 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(keys + base);
#pragma unroll
        for (int q = 0; q < RADIX_ITEMS / 4; ++q) {
            const uint4 v = src[q];
            k[4 * q] = v.x; k[4 * q + 1] = v.y; k[4 * q + 2] = v.z; k[4 * q + 3] = v.w;
        }
        nk = RADIX_ITEMS;
    } else {
#pragma unroll
        for (int q = 0; q < RADIX_ITEMS; ++q) k[q] = base + q < n ? keys[base + q] : 0u;
        nk = base < n ? (int)(n - base) : 0;
    }
    uint32_t cur = 0xffffffffu, run = 0;
#pragma unroll
    for (int q = 0; q < RADIX_ITEMS; ++q) {
        if (q < nk) {
            const uint32_t d = ((k[q] - key_sub) >> shift) & mask;
            if (d != cur) {
                if (run) atomicAdd(&cnt[w][cur], run);
                cur = d;
                run = 0;
            }
            ++run;
        }
    }
    if (run) atomicAdd(&cnt[w][cur], run);
    __syncthreads();
    for (uint32_t d = threadIdx.x; d < nbins; d += RADIX_THREADS) {
        uint32_t s = 0;
#pragma unroll
        for (int q = 0; q < RADIX_WARPS; ++q) s += cnt[q][d];
        hist[(int64_t)d * nblocks + blockIdx.x] = s;
    }
}

// key_sub: subtracted from every key read, and the rebased key written (first pass of a rebased
// sort); vals_in NULL: the values are the keys' indices
__global__ void __launch_bounds__(RADIX_THREADS) k_radix_scatter(const uint32_t *__restrict__ keys_in,
                                                                 const uint32_t *__restrict__ vals_in, int64_t n,
                                                                 int shift, int nbits, uint32_t key_sub,
                                                                 const uint32_t *__restrict__ offsets,
                                                                 int64_t nblocks, uint32_t *__restrict__ keys_out,
                                                                 uint32_t *__restrict__ vals_out) {
    chain_enter();
    // ranks are stable: warp-striped runs of 32 keys in index order, counted per warp and digit;
    // the block's keys are then laid out by digit in shared memory so that each digit's run is
    // written to its global bucket with consecutive addresses
    __shared__ uint32_t cnt[RADIX_WARPS][1 << RADIX_MAX_BITS];
    __shared__ uint32_t gbase[1 << RADIX_MAX_BITS];
    __shared__ uint32_t lbase[1 << RADIX_MAX_BITS];
    __shared__ uint32_t skey[RADIX_TILE];
    __shared__ uint32_t sval[RADIX_TILE];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nbins = 1u << nbits, mask = nbins - 1;
    for (int i = threadIdx.x; i < RADIX_WARPS * (1 << RADIX_MAX_BITS); i += RADIX_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * RADIX_TILE;
    const int64_t seg = tile0 + (int64_t)w * (RADIX_ITEMS * 32);
    const uint32_t lt = lanemask_lt();
    uint32_t key[RADIX_ITEMS], val[RADIX_ITEMS], dr[RADIX_ITEMS];
#pragma unroll
    for (int j = 0; j < RADIX_ITEMS; ++j) {
        const int64_t idx = seg + j * 32 + lane;
        const bool valid = idx < n;
        key[j] = valid ? keys_in[idx] - key_sub : 0u;
        val[j] = valid ? (vals_in ? vals_in[idx] : (uint32_t)idx) : 0u;
        const uint32_t d = valid ? (key[j] >> shift) & mask : 0xffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t base = 0;
        if (valid) base = cnt[w][d];
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[w][d] = base + __popc(peers);
        __syncwarp();
        dr[j] = valid ? ((base + __popc(peers & lt)) << 9) | d : 0xffffffffu;
    }
    __syncthreads();
    // per digit: offsets of the warps inside the block's run of that digit, and the run's total
    uint32_t total = 0;
    const uint32_t d_own = threadIdx.x;  // RADIX_THREADS == 256 digits
    if (d_own < nbins) {
#pragma unroll
        for (int q = 0; q < RADIX_WARPS; ++q) {
            const uint32_t c = cnt[q][d_own];
            cnt[q][d_own] = total;
            total += c;
        }
        gbase[d_own] = offsets[(int64_t)d_own * nblocks + blockIdx.x];
    }
    // block-local start of every digit's run: exclusive scan of the totals over the digits
    {
        uint32_t x = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ uint32_t wsum[RADIX_WARPS];
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        uint32_t wpre = 0;
#pragma unroll
        for (int q = 0; q < RADIX_WARPS; ++q)
            if (q < w) wpre += wsum[q];
        lbase[d_own] = wpre + x - total;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RADIX_ITEMS; ++j) {
        if (dr[j] == 0xffffffffu) continue;
        const uint32_t d = dr[j] & 511u, r = dr[j] >> 9;
        const uint32_t at = lbase[d] + cnt[w][d] + r;
        skey[at] = key[j];
        sval[at] = val[j];
    }
    __syncthreads();
    const int nvalid = (int)min((int64_t)RADIX_TILE, n - tile0);
    for (int i = threadIdx.x; i < nvalid; i += RADIX_THREADS) {
        const uint32_t k = skey[i];
        const uint32_t d = (k >> shift) & mask;
        const uint32_t dst = gbase[d] + ((uint32_t)i - lbase[d]);
        if (!checked((int64_t)dst < n, CS_BAD_SORT_SLOT)) continue;
        keys_out[dst] = k;
        vals_out[dst] = sval[i];
    }
}

// ---- pairs ----------------------------------------------------------------------------------
__global__ void k_depth_sort_input(const uint32_t *__restrict__ depth_keys, int64_t n, uint32_t key_min,
                                   uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        keys_out[i] = depth_keys[i] - key_min;
        vals_out[i] = (uint32_t)i;
    }
}

__device__ __forceinline__ int view_of_record(const ViewDesc *__restrict__ views, int n_views, uint32_t r) {
    int v = 0;
    while (v + 1 < n_views && (int64_t)r >= views[v + 1].rec_base) ++v;
    return v;
}

__global__ void k_view_keys(const ViewDesc *__restrict__ views, int n_views, const uint32_t *__restrict__ sorted,
                            int64_t n, uint32_t *__restrict__ keys) {
    chain_enter();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) keys[j] = (uint32_t)view_of_record(views, n_views, sorted[j]);
}

// pair key = view << local_bits | tile index within the view (row major)
// Emits the pairs of record sorted[j] at offsets[j]: every tile of its rectangle when all are kept
// (count == area), else the tiles the exact test keeps, tested by the thread itself for small
// rectangles and by the whole warp, 32 tiles at a time, for large ones.
// bit 2 q + c: the pixel box bb holds a pixel centre of the 8x4 block in column c, row q of tile
// (tx, ty), with the blend gather's test and values
__device__ __forceinline__ uint32_t block_mask(const float4 &bb, uint32_t tx, uint32_t ty) {
    uint32_t m = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float x0 = (float)(tx * TILE + 8 * c) + 0.5f, x1 = x0 + 7.0f;
        if (bb.z < x0 || bb.x > x1) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float y0 = (float)(ty * TILE + 4 * q) + 0.5f, y1 = y0 + 3.0f;
            if (!(bb.w < y0 || bb.y > y1)) m |= 1u << (2 * q + c);
        }
    }
    return m;
}

constexpr int EMIT_THREADS = 256;  // records per emit block

// position of the set bit of m that has k set bits below it (k < popc(m))
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t k) {
    uint32_t pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const uint32_t low = (uint32_t)__popc(m & ((1u << w) - 1u));
        if (k >= low) {
            k -= low;
            m >>= w;
            pos += (uint32_t)w;
        }
    }
    return pos;
}

__global__ void k_emit(const ViewDesc *__restrict__ views, int n_views, const uint32_t *__restrict__ sorted,
                       const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ counts,
                       const uint2 *__restrict__ rects, const float4 *__restrict__ records,
                       const float *__restrict__ radii, const uint32_t *__restrict__ kept,
                       const float4 *__restrict__ bboxes, int64_t n_records, int local_bits, int mask_shift,
                       uint32_t *__restrict__ keys, uint32_t *__restrict__ vals, uint32_t n_pairs) {
    // the block mask of tile (tx, ty) for box bb, at its place in the key (0 without masks)
    auto mask_bits = [&](const float4 &bb, uint32_t tx, uint32_t ty) -> uint32_t {
        return mask_shift ? block_mask(bb, tx, ty) << mask_shift : 0u;
    };
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint32_t r = 0, cnt = 0, area = 0, o = 0xffffffffu, hi = 0, tiles_x = 0, km = 0;
    uint2 rc = make_uint2(0, 0);
    float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < n_records) {
        r = sorted[j];
        cnt = counts[r];
        o = offsets[j];
        if (cnt != 0) {
            rc = rects[r];
            if (mask_shift) bb = bboxes[r];
            area = ((rc.x >> 16) - (rc.x & 0xffffu) + 1) * ((rc.y >> 16) - (rc.y & 0xffffu) + 1);
            const int v = view_of_record(views, n_views, r);
            hi = (uint32_t)v << local_bits;
            tiles_x = (uint32_t)views[v].tiles_x;
            if (cnt != area && area <= 32u) km = kept[r];
        }
    }
    const bool full = cnt != 0 && cnt == area;                     // every tile of the rectangle
    const bool masked = cnt != 0 && cnt != area && area <= 32u;     // the kept tiles of a small one
    const bool coop = cnt != 0 && cnt != area && area > 32u;        // a large rectangle, tested here
    // The block's records, consecutive in depth order, own the contiguous output range from its
    // first offset to the end of its last record.  The pairs of full and masked rectangles are
    // written by all threads of the block with consecutive addresses, output p belonging to the
    // last record whose offset is <= p (offsets do not decrease; threads past the end hold
    // 0xffffffff), so that a record with many tiles is spread over the block.  The k-th pair of a
    // rectangle is its k-th tile in row-major order (full), or the tile of its k-th kept bit
    // (masked), the order in which the preprocess counted them.
    __shared__ uint32_t s_o[EMIT_THREADS], s_r[EMIT_THREADS], s_rx[EMIT_THREADS], s_ry[EMIT_THREADS];
    __shared__ uint32_t s_hi[EMIT_THREADS], s_txs[EMIT_THREADS], s_km[EMIT_THREADS];
    __shared__ uint8_t s_kind[EMIT_THREADS];
    __shared__ float4 s_bb[EMIT_THREADS];
    __shared__ uint32_t s_end[EMIT_THREADS / 32];
    s_o[threadIdx.x] = o;
    s_r[threadIdx.x] = r;
    s_rx[threadIdx.x] = rc.x;
    s_ry[threadIdx.x] = rc.y;
    s_hi[threadIdx.x] = hi;
    s_txs[threadIdx.x] = tiles_x;
    s_km[threadIdx.x] = km;
    s_kind[threadIdx.x] = full ? 1 : masked ? 2 : 0;
    s_bb[threadIdx.x] = bb;
    const uint32_t wend = __reduce_max_sync(0xffffffffu, j < n_records ? o + cnt : 0u);
    if (lane == 0) s_end[threadIdx.x >> 5] = wend;
    __syncthreads();
    uint32_t be = 0;
#pragma unroll
    for (int q = 0; q < EMIT_THREADS / 32; ++q) be = max(be, s_end[q]);
    for (uint32_t p = s_o[0] + threadIdx.x; p < be; p += EMIT_THREADS) {
        int sr = 0;
#pragma unroll
        for (int step = EMIT_THREADS / 2; step >= 1; step >>= 1)
            if (s_o[sr + step] <= p) sr += step;
        const int kind = s_kind[sr];
        if (kind == 0 || !checked(p < n_pairs, CS_BAD_PAIR_SLOT)) continue;
        const uint32_t rx = s_rx[sr], ry = s_ry[sr];
        const uint32_t k = p - s_o[sr], wd = (rx >> 16) - (rx & 0xffffu) + 1;
        const uint32_t q = kind == 2 ? nth_set_bit(s_km[sr], k) : k;
        const uint32_t ty = (ry & 0xffffu) + q / wd, tx = (rx & 0xffffu) + q % wd;
        keys[p] = mask_bits(s_bb[sr], tx, ty) | s_hi[sr] | (ty * s_txs[sr] + tx);
        vals[p] = s_r[sr];
    }
    uint32_t pending = __ballot_sync(0xffffffffu, coop);
    while (pending) {  // large rectangles: the warp tests 32 tiles at a time, kept ones in row-major order
        const int src = __ffs(pending) - 1;
        pending &= pending - 1;
        const uint32_t rs = __shfl_sync(0xffffffffu, r, src), hs = __shfl_sync(0xffffffffu, hi, src);
        const uint32_t txs = __shfl_sync(0xffffffffu, tiles_x, src);
        const uint32_t rx = __shfl_sync(0xffffffffu, rc.x, src), ry = __shfl_sync(0xffffffffu, rc.y, src);
        uint32_t os = __shfl_sync(0xffffffffu, o, src);
        float4 bs;
        bs.x = __shfl_sync(0xffffffffu, bb.x, src);
        bs.y = __shfl_sync(0xffffffffu, bb.y, src);
        bs.z = __shfl_sync(0xffffffffu, bb.z, src);
        bs.w = __shfl_sync(0xffffffffu, bb.w, src);
        float w[REC_WORDS];
        const float4 *rec = records + (size_t)rs * (REC_WORDS / 4);
#pragma unroll
        for (int q = 0; q < REC_WORDS / 4; ++q) {
            const float4 f = rec[q];
            w[4 * q] = f.x; w[4 * q + 1] = f.y; w[4 * q + 2] = f.z; w[4 * q + 3] = f.w;
        }
        const int T = (int)hull_pack_count(__float_as_uint(w[R_HULL]));
        const float rk = radii[rs];
        const uint32_t x0 = rx & 0xffffu, y0 = ry & 0xffffu;
        const uint32_t wd = (rx >> 16) - x0 + 1, ar = wd * ((ry >> 16) - y0 + 1);
        for (uint32_t base = 0; base < ar; base += 32) {
            const uint32_t q = base + (uint32_t)lane;
            const uint32_t tx = x0 + q % wd, ty = y0 + q / wd;
            const bool keep = q < ar && tile_kept(w + R_LINES, T, w[R_AX], w[R_AY], rk, (int)tx, (int)ty);
            const uint32_t ball = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const uint32_t at = os + (uint32_t)__popc(ball & ((1u << lane) - 1u));
                if (checked(at < n_pairs, CS_BAD_PAIR_SLOT)) {
                    keys[at] = mask_bits(bs, tx, ty) | hs | (ty * txs + tx);
                    vals[at] = rs;
                }
            }
            os += (uint32_t)__popc(ball);
        }
    }
}

// [start, end) of every (view, tile) group of the sorted pairs, stored at the global tile index
// RANGE_ITEMS consecutive sorted keys per thread (two 16-byte loads), each compared with its
// neighbours; only the first and last pair of a (view, tile) group look up the view and write.
constexpr int RANGE_ITEMS = 8;
__global__ void k_ranges(const uint32_t *__restrict__ keys, int64_t n, const ViewDesc *__restrict__ views,
                         int local_bits, uint32_t key_mask, uint2 *__restrict__ ranges, int n_views,
                         int64_t n_tiles) {
    const int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * RANGE_ITEMS;
    if (i0 >= n) return;
    uint32_t k[RANGE_ITEMS + 2];  // keys i0 - 1 .. i0 + RANGE_ITEMS (masked)
    if (i0 + RANGE_ITEMS <= n && (reinterpret_cast<uintptr_t>(keys) & 15) == 0) {
        const uint4 a = reinterpret_cast<const uint4 *>(keys + i0)[0], b = reinterpret_cast<const uint4 *>(keys + i0)[1];
        k[1] = a.x; k[2] = a.y; k[3] = a.z; k[4] = a.w; k[5] = b.x; k[6] = b.y; k[7] = b.z; k[8] = b.w;
    } else {
#pragma unroll
        for (int q = 0; q < RANGE_ITEMS; ++q) k[q + 1] = i0 + q < n ? keys[i0 + q] : 0u;
    }
    k[0] = i0 > 0 ? keys[i0 - 1] : 0u;
    k[RANGE_ITEMS + 1] = i0 + RANGE_ITEMS < n ? keys[i0 + RANGE_ITEMS] : 0u;
#pragma unroll
    for (int q = 0; q < RANGE_ITEMS + 2; ++q) k[q] &= key_mask;
#pragma unroll
    for (int q = 0; q < RANGE_ITEMS; ++q) {
        const int64_t i = i0 + q;
        if (i >= n) break;
        const uint32_t kc = k[q + 1];
        const bool start = i == 0 || k[q] != kc, end = i == n - 1 || k[q + 2] != kc;
        if (!(start || end)) continue;
        if (!checked((int64_t)(kc >> local_bits) < n_views, CS_BAD_TILE)) continue;
        const uint32_t g = views[kc >> local_bits].tile_base + (kc & ((1u << local_bits) - 1u));
        if (!checked((int64_t)g < n_tiles, CS_BAD_TILE)) continue;
        if (start) ranges[g].x = (uint32_t)i;
        if (end) ranges[g].y = (uint32_t)(i + 1);
    }
}

}  // namespace

size_t scan_tmp_words(int64_t n) { return (size_t)((n + SCAN_TILE - 1) / SCAN_TILE) + 1; }

// Launches a chain kernel; with pdl, as a programmatic dependent of the kernel before it in the
// stream (only when that stream operation is a chain kernel: the kernel's wait then covers it).
template <typename... Exp, typename... Act>
static cudaError_t launch_chain(bool pdl, void (*kernel)(Exp...), unsigned grid, unsigned block, cudaStream_t s,
                                Act &&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Act>(args)...);
}

cudaError_t launch_exclusive_scan(const uint32_t *in, const uint32_t *gather, uint32_t *out, int64_t n,
                                  unsigned long long *total_dev, unsigned long long *tmp, cudaStream_t s,
                                  bool pdl_first) {
    if (n <= 0) {
        if (total_dev) return fill_words(total_dev, 0u, sizeof(unsigned long long), s);
        return cudaSuccess;
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    cudaError_t e = launch_chain(pdl_first, k_scan_reduce, (unsigned)nb, SCAN_THREADS, s, in, gather, n, tmp);
    if (e != cudaSuccess) return e;
    if (nb <= SCAN_INLINE_BLOCKS) {
        e = launch_chain(true, k_scan_down<true>, (unsigned)nb, SCAN_THREADS, s, in, gather, n,
                         (const unsigned long long *)tmp, out, total_dev);
        count_launches(2);
    } else {
        e = launch_chain(true, k_scan_spine, 1u, SPINE_THREADS, s, tmp, nb, total_dev);
        if (e == cudaSuccess)
            e = launch_chain(true, k_scan_down<false>, (unsigned)nb, SCAN_THREADS, s, in, gather, n,
                             (const unsigned long long *)tmp, out, (unsigned long long *)nullptr);
        count_launches(3);
    }
    return e;
}

size_t radix_tmp_words(int64_t n) {
    const int64_t nb = (n + RADIX_TILE - 1) / RADIX_TILE;
    return (size_t)(nb * (1 << RADIX_MAX_BITS) * 2);
}

cudaError_t radix_sort_pairs(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, int64_t n,
                             int bits, uint32_t *tmp, unsigned long long *scan_tmp, bool *result_in_b,
                             cudaStream_t s, const uint32_t *first_keys, uint32_t first_key_sub, int bit_begin,
                             bool pdl_first) {
    *result_in_b = false;
    if (n <= 1 || bits <= bit_begin) return cudaSuccess;
    const int64_t nb = (n + RADIX_TILE - 1) / RADIX_TILE;
    const int passes = (bits - bit_begin + RADIX_MAX_BITS - 1) / RADIX_MAX_BITS;
    uint32_t *hist = tmp;
    uint32_t *offs = tmp + nb * (1 << RADIX_MAX_BITS);
    const uint32_t *kin = first_keys ? first_keys : keys_a;
    const uint32_t *vin = first_keys ? nullptr : vals_a;
    uint32_t *kout = keys_b, *vout = vals_b;
    int shift = bit_begin;
    for (int p = 0; p < passes; ++p) {
        const int w = (bits - shift + (passes - p) - 1) / (passes - p);  // spread the bits evenly
        const int64_t nh = (int64_t)(1 << w) * nb;
        const uint32_t sub = (p == 0 && first_keys) ? first_key_sub : 0u;
        cudaError_t e = launch_chain(p > 0 || pdl_first, k_radix_upsweep, (unsigned)nb, RADIX_THREADS, s, kin, n, shift,
                                     w, sub, hist, nb);
        if (e == cudaSuccess) e = launch_exclusive_scan(hist, nullptr, offs, nh, nullptr, scan_tmp, s, true);
        if (e == cudaSuccess)
            e = launch_chain(true, k_radix_scatter, (unsigned)nb, RADIX_THREADS, s, kin, vin, n, shift, w, sub,
                             (const uint32_t *)offs, nb, kout, vout);
        if (e != cudaSuccess) return e;
        count_launches(2);
        shift += w;
        // the next pass reads what this one wrote and writes the other buffer (never first_keys)
        uint32_t *next_k = kout == keys_b ? keys_a : keys_b, *next_v = vout == vals_b ? vals_a : vals_b;
        kin = kout;
        vin = vout;
        kout = next_k;
        vout = next_v;
        *result_in_b = !*result_in_b;
    }
    return cudaGetLastError();
}

cudaError_t launch_depth_sort_input(const uint32_t *depth_keys, int64_t n, uint32_t key_min, uint32_t *keys_out,
                                    uint32_t *vals_out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_depth_sort_input<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(depth_keys, n, key_min, keys_out, vals_out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_view_keys(const ViewDesc *views_dev, int n_views, const uint32_t *sorted_records, int64_t n,
                             uint32_t *keys, cudaStream_t s, bool pdl) {
    if (n <= 0) return cudaSuccess;
    const cudaError_t e = launch_chain(pdl, k_view_keys, (unsigned)((n + 255) / 256), 256u, s, views_dev, n_views,
                                       sorted_records, n, keys);
    count_launches(1);
    return e;
}

cudaError_t launch_emit_pairs(const ViewDesc *views_dev, int n_views, const uint32_t *sorted_records,
                              const uint32_t *offsets, const uint32_t *counts, const uint2 *rects,
                              const float4 *records, const float *radii, const uint32_t *kept,
                              const float4 *bboxes, int64_t n_records, int local_bits, int mask_shift,
                              uint32_t *pair_keys, uint32_t *pair_vals, cudaStream_t s, uint32_t n_pairs) {
    if (n_records <= 0) return cudaSuccess;
    if (mask_shift < 0 || (mask_shift > 0 && mask_shift + BLOCK_MASK_BITS > 32)) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((n_records + EMIT_THREADS - 1) / EMIT_THREADS);
    k_emit<<<blocks, EMIT_THREADS, 0, s>>>(views_dev, n_views, sorted_records, offsets, counts, rects, records, radii,
                                           kept, bboxes, n_records, local_bits, mask_shift, pair_keys, pair_vals,
                                           n_pairs);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tile_ranges(const uint32_t *pair_keys, int64_t n_pairs, const ViewDesc *views_dev, int local_bits,
                               int mask_shift, uint2 *ranges, int64_t n_tiles, cudaStream_t s, int n_views) {
    cudaError_t e = fill_words(ranges, 0u, sizeof(uint2) * (size_t)n_tiles, s);
    if (e != cudaSuccess || n_pairs <= 0) return e;
    const uint32_t key_mask = mask_shift ? (1u << mask_shift) - 1u : 0xffffffffu;
    const int64_t threads = (n_pairs + RANGE_ITEMS - 1) / RANGE_ITEMS;
    k_ranges<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(pair_keys, n_pairs, views_dev, local_bits, key_mask,
                                                               ranges, n_views, n_tiles);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t take_status_sort(unsigned *bits, cudaStream_t s) {
#if CS_CHECKED
    unsigned v = 0;
    const unsigned zero = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_status_sort, sizeof v, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_status_sort, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) *bits |= v;
    return e;
#else
    (void)bits;
    (void)s;
    return cudaSuccess;
#endif
}

}  // namespace cs
