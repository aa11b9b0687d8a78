// Internal definitions shared by the CUDA sources of the convex tile rasterizer (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/convex_splat.h"

namespace cs {

constexpr int KMAX = 8;    // most points per convex
constexpr int TILE = 16;   // tile edge in pixels
constexpr int REC_WORDS = 32;   // 128-byte screen record per (view, convex)
constexpr int GRAD_WORDS = 32;  // 128-byte gradient record per (view, convex)

// Screen record layout (32-bit words), written by the preprocess, read by both blends:
//   0, 1   anchor a = first hull vertex (pixels); lines below are expressed relative to it
//   2      sigma' = d^p sigma
//   3      opacity o
//   4..6   colour c (after the clamp at 0)
//   7      hull: T in bits 0-3, index of hull vertex i in bits 4+3i..6+3i
//   8+3t   A_t = kappa n_t.x          kappa = log2(e) d^p delta, so that
//   9+3t   B_t = kappa n_t.y          kappa L_t(q) = A_t (q.x - a.x) + B_t (q.y - a.y) + C_t
//   10+3t  C_t = kappa n_t . (a - v_t)
constexpr int R_AX = 0, R_AY = 1, R_SIG = 2, R_OPA = 3, R_RGB = 4, R_HULL = 7, R_LINES = 8;

// Gradient record layout: d(loss)/d(screen record quantities)
//   3t+0..2  dA_t, dB_t, dC_t     24 dsigma'    25 dopacity    26..28 dcolour
constexpr int G_SIG = 24, G_OPA = 25, G_RGB = 26;

struct ViewDesc {
    // camera
    float R[9];
    float t[3];
    float fx, fy, cx, cy, z_near;
    float campos[3];  // camera centre in world coordinates (-R^T t), for the SH direction
    int32_t width, height, tiles_x, tiles_y;
    uint32_t tile_base;  // first global tile index of this view
    int64_t rec_base;    // first record index of this view
    // scene (device)
    const void *points, *delta, *sigma, *opacity, *sh;  // elements of type `storage`
    int64_t n;
    int32_t k, sh_degree;
    int32_t activation;  // 0: delta, sigma, opacity as given; 1: exp, exp, sigmoid of the given values
    int32_t storage;     // cs_storage: float32, binary16 or bfloat16 parameters
    // outputs (device)
    float *image;     // [3][H][W]
    float *t_final;   // [H][W]
    uint32_t *n_last; // [H][W]
};

struct Settings {
    float tau, alpha_max, t_min;
    float bg[3];
    int32_t dist_mode;
    float dist_power;
    int32_t tile_test;
    int32_t tile_split;
};

__host__ __device__ inline uint32_t hull_pack_count(uint32_t packed) { return packed & 15u; }
__host__ __device__ inline int hull_pack_index(uint32_t packed, int i) { return (int)((packed >> (4 + 3 * i)) & 7u); }

// ---- launch wrappers implemented in the .cu files --------------------------------------------
// totals of a preprocess launch, accumulated with atomics into a zeroed struct: the pairs to emit
// and the range of the drawn records' depth keys (the minimum kept as the maximum of its complement
// so that all-zero bytes are the empty state)
struct PreprocessStats {
    unsigned long long pairs;
    unsigned int key_max, key_min_inv;
};

struct PreprocessOut {
    float4 *records;       // [R][8]
    uint32_t *depth_keys;  // [R]
    uint2 *rects;          // [R]
    uint32_t *counts;      // [R]
    float4 *bboxes;        // [R] pixel box (xmin, ymin, xmax, ymax) holding every pixel with alpha >= tau
    float *radii;          // [R] kappa r, the tile test's bound in record units
    uint32_t *kept;        // [R] rectangles of at most 32 tiles: bit q set when tile q (row-major in
                           // the rectangle) holds pairs of the record (after the exact tile test)
    PreprocessStats *stats;  // zeroed before the launch
};
cudaError_t launch_preprocess(const ViewDesc *views_dev, const ViewDesc *views_host, int n_views, int64_t max_n,
                              int k, const Settings &st, const PreprocessOut &out, cudaStream_t s);

struct PreprocessGrads {
    float *dpoints, *ddelta, *dsigma, *dopacity, *dsh;
    bool write = false;  // single view: write the gradients instead of adding them to the buffers
};
cudaError_t launch_preprocess_backward(const ViewDesc *views_dev, int n_views, int64_t max_n, int k, int sh_degree,
                                       int storage, const Settings &st, const float4 *records, const uint32_t *counts,
                                       const float4 *grad_records, const PreprocessGrads &g, bool atomic,
                                       cudaStream_t s);

// device-wide exclusive scan of n uint32 values (optionally gathered through idx); writes the
// 64-bit total to *total_dev.  tmp must hold scan_tmp_words(n) uint64 words.
// pdl_first (here and below): the stream operation before the call is a kernel of the sort chain,
// so the first launch may be a programmatic dependent of it.
size_t scan_tmp_words(int64_t n);
cudaError_t launch_exclusive_scan(const uint32_t *in, const uint32_t *gather_idx, uint32_t *out, int64_t n,
                                  unsigned long long *total_dev, unsigned long long *tmp, cudaStream_t s,
                                  bool pdl_first = false);

// stable LSD radix sort of (key, value) pairs on the low `bits` key bits.  Buffers a/b alternate;
// returns in *result_in_b whether the sorted data ended in the b buffers.  With first_keys, the
// input is (first_keys[i] - first_key_sub, i) instead of the a buffers (first_keys is only read; the
// sort needs bits > bit_begin then, since with no pass nothing is written).  Bits below bit_begin
// are taken as already sorted by earlier passes.
size_t radix_tmp_words(int64_t n);
cudaError_t radix_sort_pairs(uint32_t *keys_a, uint32_t *vals_a, uint32_t *keys_b, uint32_t *vals_b, int64_t n,
                             int bits, uint32_t *tmp, unsigned long long *scan_tmp, bool *result_in_b,
                             cudaStream_t s, const uint32_t *first_keys = nullptr, uint32_t first_key_sub = 0,
                             int bit_begin = 0, bool pdl_first = false);

// the depth sort's input: keys_out[i] = depth_keys[i] - key_min (mod 2^32), vals_out[i] = i.  The
// drawn records' keys then lie in [0, key_max - key_min]; undrawn records (which emit no pairs)
// take whatever low bits the subtraction leaves them
cudaError_t launch_depth_sort_input(const uint32_t *depth_keys, int64_t n, uint32_t key_min, uint32_t *keys_out,
                                    uint32_t *vals_out, cudaStream_t s);
// keys[j] = view index of record sorted_records[j]
cudaError_t launch_view_keys(const ViewDesc *views_dev, int n_views, const uint32_t *sorted_records, int64_t n,
                             uint32_t *keys, cudaStream_t s, bool pdl = false);
// pair key = view << local_bits | tile index within the view, and, when mask_shift > 0, the pair's
// block mask << mask_shift: bit 2 q + c set when the record's pixel box holds a pixel centre of the
// tile's 8x4 block in column c, row q (the blocks of the forward blend's warps).  The tile sort
// orders local_bits only, so the mask bits travel with their pair.
constexpr int BLOCK_MASK_BITS = 8;
cudaError_t launch_emit_pairs(const ViewDesc *views_dev, int n_views, const uint32_t *sorted_records,
                              const uint32_t *offsets, const uint32_t *counts, const uint2 *rects,
                              const float4 *records, const float *radii, const uint32_t *kept,
                              const float4 *bboxes, int64_t n_records, int local_bits, int mask_shift,
                              uint32_t *pair_keys, uint32_t *pair_vals, cudaStream_t s,
                              uint32_t n_pairs = 0xffffffffu);
cudaError_t launch_tile_ranges(const uint32_t *pair_keys, int64_t n_pairs, const ViewDesc *views_dev, int local_bits,
                               int mask_shift, uint2 *ranges, int64_t n_tiles, cudaStream_t s, int n_views);

// ---- checked builds ---------------------------------------------------------------------------
// Built with -DCS_CHECKED=1, the kernels test every index that an inconsistent upstream value could
// send out of bounds before using it; a failed test skips (or clamps) the access and sets a bit in
// its translation unit's device status word, and the entry points read and clear those words once
// their stream has finished, returning CS_ERR_DEVICE.  Transient buffers are also filled with 0xff
// bytes (NaN as float) when they are taken from the pool, so that reading a buffer before it is
// written changes the results.  Production builds compile all of it out.
#ifndef CS_CHECKED
#define CS_CHECKED 0
#endif
enum : uint32_t {
    CS_BAD_RANGE = 1u,      // a tile's pair range outside the pair list
    CS_BAD_RECORD = 2u,     // a pair's record index beyond the records
    CS_BAD_HULL = 4u,       // a record's hull line count outside 3..K
    CS_BAD_PAIR_SLOT = 8u,  // an emitted pair beyond the pair list
    CS_BAD_TILE = 16u,      // a tile index beyond the tiles
    CS_BAD_SORT_SLOT = 32u  // a radix-sort destination beyond the items
};
// OR into *bits, and clear, the status words of the blend kernels / of the sort, emission and
// range kernels, after the work enqueued on s so far (synchronises s; no-ops in production builds)
cudaError_t take_status_blend(unsigned *bits, cudaStream_t s);
cudaError_t take_status_sort(unsigned *bits, cudaStream_t s);

struct BlendArgs {
    const ViewDesc *views;
    int n_views;
    const uint2 *ranges;
    const uint32_t *pair_vals;
    const float4 *records;
    const float4 *bboxes;
    Settings st;
    uint32_t n_tiles;
    int k;  // points per convex: at most k hull lines per record
    const uint32_t *pair_keys;  // with block masks when mask_shift > 0
    int mask_shift;             // 0: no masks, the gather tests the records' pixel boxes
    uint32_t tile_offset = 0;   // global index of the launch's first tile (its tiles: n_tiles from there)
    uint32_t n_pairs = 0xffffffffu;    // pair-list length and record count: bounds of the checked
    uint32_t n_records = 0xffffffffu;  // builds' index tests (all ones: unknown)
    // tile split (split > 0 pairs per chunk): work items (tile, chunk) of the chunked launches,
    // heavy tiles (tile, first slot) of the merge, each tile's first slot, the chunk states
    // launch order of the tiles (PLAIN mode; NULL: tile index order): longest pair lists first
    const uint32_t *tile_order = nullptr;
    // one persistent launch over the tiles of all views (view_flags != NULL; the tile order view by
    // view): each CTA takes the next tile of tile_order from *queue, counts the tiles it finishes
    // per view in view_tiles_done (both zero when the launch starts) and, on a view's last tile,
    // stores flag_value into view_flags[view] (mapped host memory) once the view's image is written
    uint32_t *queue = nullptr;
    uint32_t *view_tiles_done = nullptr;
    uint32_t *view_flags = nullptr;
    uint32_t flag_value = 0;
    uint32_t split = 0;
    const uint2 *split_items = nullptr;
    uint32_t n_items = 0;
    const uint2 *split_heavy = nullptr;
    uint32_t n_heavy = 0;
    const uint32_t *split_slot = nullptr;
    float *chunk_state = nullptr;
};
// Tile split planning: per tile, the chunks of a heavy tile (more than `split` pairs; 0 for a
// light tile) into heavy[], 1 for a light tile into light[], and the number of heavy tiles added
// to *n_heavy_tiles (zeroed by the caller)
cudaError_t launch_split_count(const uint2 *ranges, uint32_t n_tiles, uint32_t split, uint32_t *heavy, uint32_t *light,
                               unsigned int *n_heavy_tiles, cudaStream_t s);
// work items: heavy chunks first, at slot heavy_base[g] + chunk, then light tiles at
// n_slots + light_base[g]; heavy tiles listed (order free) with their first slot; per tile its
// first slot (0xffffffff for a light tile).  *heavy_fill zeroed by the caller.
cudaError_t launch_split_items(const uint2 *ranges, uint32_t n_tiles, uint32_t split, const uint32_t *heavy_base,
                               const uint32_t *light_base, uint32_t n_slots, uint2 *items, uint2 *heavy_list,
                               unsigned int *heavy_fill, uint32_t *slot_of_tile, cudaStream_t s);
constexpr int SPLIT_STATE_FLOATS = 5 * 256;  // per chunk slot: 5 words for each pixel of a 16x16 tile
// Launch order of the blend CTAs: the tiles by decreasing floor(log2(pairs + 1)) (order within a
// class free), so that the longest pair lists start first and do not trail the grid; by_view: view
// by view in view order (at most MAX_ORDER_VIEWS views), longest lists first within each.  One
// launch of one CTA; order: n_tiles words.  Each tile's outputs do not depend on when its CTA
// runs.  The kernel also zeroes the n_zero words at zero_words (the persistent blend's counters).
constexpr int TILE_ORDER_CLASSES = 32;
constexpr int MAX_ORDER_VIEWS = 32;
cudaError_t launch_tile_order(const uint2 *ranges, uint32_t n_tiles, uint32_t *order, const ViewDesc *views,
                              int n_views, bool by_view, uint32_t *zero_words, int n_zero, cudaStream_t s);
// counts: NULL for the production kernels, else 6 zeroed uint64 counters for the instrumented ones
cudaError_t launch_blend_forward(const BlendArgs &a, cudaStream_t s, unsigned long long *counts = nullptr);
cudaError_t launch_blend_backward(const BlendArgs &a, const float *dL_dimage, int64_t image_stride,
                                  float4 *grad_records, cudaStream_t s, unsigned long long *counts = nullptr);

// Small transfers done by kernels, never by a copy engine (transfer.cu): the words of p (4-byte
// aligned, bytes a multiple of 4) set to v; n view descriptors copied from host memory (read when
// the call is made) to device memory; `words` 32-bit words copied from device memory to pinned
// host memory mapped into the device's address space (visible to the host once the stream has
// reached the end of the kernel)
cudaError_t fill_words(void *p, uint32_t v, size_t bytes, cudaStream_t s);
cudaError_t put_views(ViewDesc *dst, const ViewDesc *src, int n, cudaStream_t s);
cudaError_t publish_words(const void *src, void *dst_host_mapped, int words, cudaStream_t s);

// process-wide count of kernel launches made by the library
void count_launches(int n);

}  // namespace cs
