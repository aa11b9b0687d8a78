// Per-tile blending of the convex tile rasterizer, forward and backward.
//
// Forward: each warp an 8x4 pixel block, each thread one pixel, 128 threads per half tile (16x8;
// 256 per 16x16 tile in the tile-split, counting and persistent variants); backward: 128 threads
// per tile, each warp an 8x8 block, each thread two pixels (rows r and r + 4).  The warps work
// independently (no CTA barrier).  A warp walks the tile's depth-ordered pairs, keeping those
// whose record's pixel box reaches its block (the block-mask bit carried in the pair key, or the
// box itself), 32 at a time, and stages their records in its shared-memory slice (the forward
// copies the 32 records with coalesced cp.async, four whole records per instruction, and each
// lane then rewrites its own in place; the backward's lanes load theirs with vector loads): each
// record is re-expressed relative to the warp's block origin so that every line is two FMAs per
// pixel, and tested for whether any pixel of the block can pass the line pre-test; the warp then
// evaluates only the records of the resulting ballot.  Per pixel and convex (Eq. S1, S2 and 5):
//     s_t  = log2(e) d delta L_t(q)                     (T lines, 2 FMA each)
//     phi2 = max_t s_t + log2 sum_t 2^(s_t - max)       (= log2(e) phi)
//     I    = 1 / (1 + 2^(d sigma phi2))                 (= Sigmoid(-d sigma phi))
//     alpha = min(alpha_max, o I); skip if alpha < tau; C += T alpha c; T *= 1 - alpha
// A pair whose largest line value already forces alpha < tau is skipped without any
// transcendental (phi >= max_t s_t).  A warp leaves its loop once every pixel of its block has
// its transmittance below t_min.
//
// The backward walks each tile's list in reverse from the last contributor of each pixel,
// recovering T before a pair as T_after / (1 - alpha) and carrying, per pixel, the colour seen
// behind the pair only through its product with dL/dC (the one scalar dL/dalpha needs), and
// accumulates d(loss)/d(record) per convex: the 3K + 5 per-pixel terms are summed across the warp
// by a reduce-scatter (16 + 8 words, 25 shuffles at K = 6, lane l ends with word l) and added to
// the convex's gradient record by one coalesced atomic instruction per (warp, record).
#include "cs_common.cuh"

#include <atomic>

namespace cs {
namespace {

#if CS_CHECKED
__device__ unsigned int g_status_blend;  // bits of the failed index tests of the blend kernels
__device__ __forceinline__ bool checked(bool ok, unsigned bit) {
    if (!ok) atomicOr(&g_status_blend, bit);
    return ok;
}
#else
__device__ __forceinline__ bool checked(bool ok, unsigned) { return true; }
#endif

constexpr int FWD_THREADS = 256;  // forward: 8 warps per tile, a warp an 8x4 block, a lane one pixel
constexpr int BWD_THREADS = 128;  // backward: 4 warps per tile, a warp an 8x8 block, a lane rows r, r + 4
// staged record (one per lane of a warp), SREC<K> float4:
//   [0] = (sigma', pre-test bound, o, T)   [1] = (r, g, b, record index)
//   [2] = (block origin minus anchor vertex: x, y, -, -)
//   [3 + t] = (A_t, B_t, C_t relative to the upper 8x4 block origin, C_t relative to the lower one)
// The forward's 8x4 blocks and the backward's two 8x4 halves of an 8x8 block are re-based to the
// same origins, so both kernels evaluate every pair with identical binary32 values.
template <int K>
constexpr int SREC = 3 + K;
// 16-byte chunks of a screen record that hold its header and K lines
template <int K>
constexpr int REC_CHUNKS = (R_LINES + 3 * K + 3) / 4;
// a warp's staging buffer, in float4: the 32 raw records (128 B each) land there first, then each
// lane re-writes its own record in the staged form over them
template <int K>
constexpr int STAGE_F4 = 32 * (SREC<K> > REC_WORDS / 4 ? SREC<K> : REC_WORDS / 4);
constexpr float LN2 = 0.6931471805599453f;

__device__ __forceinline__ void cp_async_cg16(void *dst, const void *src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;\n" ::: "memory");
}

// Copies the screen records of the nh gathered pairs (slots sidx[0..nh)) into the warp's staging
// buffer with coalesced 16-byte cp.async: one instruction moves four whole records, eight lanes
// per record, chunk c of the record in slot s landing at float4 8 s + (c ^ (s & 7)) (the XOR
// spreads the 32 records' chunk c over all banks for the per-lane reads that follow).  Returns
// this lane's record index (lane < nh).  The copies are complete and visible to the whole warp
// on return.
template <int K>
__device__ __forceinline__ uint32_t copy_records(float4 *buf, const float4 *__restrict__ records,
                                                 const uint32_t *__restrict__ pair_vals, const uint32_t *sidx, int nh,
                                                 int lane, uint32_t n_records) {
    uint32_t r = lane < nh ? __ldg(pair_vals + sidx[lane]) : 0u;
    if (!checked(r < n_records, CS_BAD_RECORD)) r = 0;
    const int c = lane & 7;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int slot = 4 * k + (lane >> 3);
        const uint32_t rs = __shfl_sync(0xffffffffu, r, slot);
        if (slot < nh && c < REC_CHUNKS<K>)
            cp_async_cg16(buf + 8 * slot + (c ^ (slot & 7)), records + (size_t)rs * (REC_WORDS / 4) + c);
    }
    cp_async_commit_wait();
    __syncwarp();
    return r;
}

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Stage record r, whose raw copy sits in the staging buffer at slot `lane` (see copy_records), for
// the pixel block of 8 x ROWS pixels whose first pixel centre is (ox + 0.5, oy + 0.5) in image
// coordinates (ROWS = 4: one 8x4 block; ROWS = 8: two stacked 8x4 blocks with origins oy and
// oy + 4), writing the staged form into the same buffer at slot `lane`.  Every lane of the warp
// calls it (lanes at or beyond nh stage nothing).  Returns false when no pixel of the block can
// pass the line pre-test: for some line, its smallest value over the block's pixel centres exceeds
// the bound (with a margin for the per-pixel rounding).
template <int ROWS, int K>
__device__ __forceinline__ bool stage_record(float4 *buf, int lane, int nh, uint32_t r, float ox, float oy,
                                             const Settings &st) {
    // the raw record of this lane, read in full before any lane overwrites the buffer
    const float4 *raw = buf + 8 * lane;
    const int sw = lane & 7;
    float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), h1 = h0;
    float L[3 * K + 3];
    if (lane < nh) {
        h0 = raw[0 ^ sw];
        h1 = raw[1 ^ sw];
#pragma unroll
        for (int q = 0; q < REC_CHUNKS<K> - 2; ++q) {
            const float4 v = raw[(q + 2) ^ sw];
            L[4 * q] = v.x; L[4 * q + 1] = v.y; L[4 * q + 2] = v.z; L[4 * q + 3] = v.w;
        }
    }
    __syncwarp();
    if (lane >= nh) return false;
    float4 *dst = buf + SREC<K> * lane;
    int T = (int)hull_pack_count(__float_as_uint(h1.w));
    if (!checked(T >= 3 && T <= K, CS_BAD_HULL)) T = 0;
    const float offx = ox - h0.x, offy = oy - h0.y, offy2 = (oy + 4.0f) - h0.y;
    // pre-test: alpha < tau whenever sigma' max_t s_t > log2(o/tau - 1) (phi2 >= max_t s_t); the
    // bound is widened so that it never rejects a pair the full evaluation keeps
    float bound = __int_as_float(0x7f800000);
    if (st.tau > 0.f) {
        const float x = h0.w / st.tau - 1.0f;
        if (isfinite(x)) {
            const float b = lg2(x) * rcp(h0.z);
            bound = b + fabsf(b) * 0x1p-10f + 0x1p-10f;
        }
    }
    bool pass = true;
#pragma unroll
    for (int t = 0; t < K; ++t) {
        if (t < T) {
            const float A = L[3 * t], B = L[3 * t + 1], C = L[3 * t + 2];
            const float Cp = fmaf(A, offx, fmaf(B, offy, C));
            const float Cp2 = ROWS == 8 ? fmaf(A, offx, fmaf(B, offy2, C)) : 0.f;
            dst[3 + t] = make_float4(A, B, Cp, Cp2);
            const float margin = (fabsf(Cp) + 8.f * (fabsf(A) + fabsf(B))) * 0x1p-20f + 0x1p-20f;
            const float mn = Cp + fminf(0.5f * A, 7.5f * A) + fminf(0.5f * B, ((float)ROWS - 0.5f) * B);
            pass = pass && !(mn > bound + margin);
        } else {
            // an unused slot: a line that is -inf everywhere adds 2^-inf = 0 to the sum and never
            // wins the maximum, so every record is evaluated with K lines
            const float ninf = -__int_as_float(0x7f800000);
            dst[3 + t] = make_float4(0.f, 0.f, ninf, ninf);
        }
    }
    dst[0] = make_float4(h0.z, bound, h0.w, __int_as_float(T));
    dst[1] = make_float4(h1.x, h1.y, h1.z, __uint_as_float(r));
    dst[2] = make_float4(offx, offy, 0.f, 0.f);
    return pass;
}

// The backward's staging: each lane loads its own record r from global memory with 16-byte
// vector loads (as many as the record's hull lines need) and writes the staged form to dst, for
// the same pixel blocks and with the same values as stage_record.  (Staging through the warp's
// cp.async copies, as the forward does, costs this kernel register spills at its occupancy of
// 6 CTAs per SM and was measured slower.)  Returns the same pre-test result.
template <int ROWS, int K>
__device__ __forceinline__ bool stage_record_ldg(float4 *dst, const float4 *__restrict__ records, uint32_t r, float ox,
                                             float oy, const Settings &st) {
    const float4 *src = records + (size_t)r * (REC_WORDS / 4);
    const float4 h0 = __ldg(src), h1 = __ldg(src + 1);
    int T = (int)hull_pack_count(__float_as_uint(h1.w));
    if (!checked(T >= 3 && T <= K, CS_BAD_HULL)) T = 0;
    float L[3 * KMAX];
#pragma unroll
    for (int q = 0; q < (3 * K + 3) / 4; ++q) {
        if (4 * q < 3 * T) {
            const float4 v = __ldg(src + 2 + q);
            L[4 * q] = v.x; L[4 * q + 1] = v.y; L[4 * q + 2] = v.z; L[4 * q + 3] = v.w;
        } else {
            L[4 * q] = L[4 * q + 1] = L[4 * q + 2] = L[4 * q + 3] = 0.f;
        }
    }
    const float offx = ox - h0.x, offy = oy - h0.y, offy2 = (oy + 4.0f) - h0.y;
    // pre-test: alpha < tau whenever sigma' max_t s_t > log2(o/tau - 1) (phi2 >= max_t s_t); the
    // bound is widened so that it never rejects a pair the full evaluation keeps
    float bound = __int_as_float(0x7f800000);
    if (st.tau > 0.f) {
        const float x = h0.w / st.tau - 1.0f;
        if (isfinite(x)) {
            const float b = lg2(x) * rcp(h0.z);
            bound = b + fabsf(b) * 0x1p-10f + 0x1p-10f;
        }
    }
    bool pass = true;
#pragma unroll
    for (int t = 0; t < K; ++t) {
        if (t < T) {
            const float A = L[3 * t], B = L[3 * t + 1], C = L[3 * t + 2];
            const float Cp = fmaf(A, offx, fmaf(B, offy, C));
            const float Cp2 = ROWS == 8 ? fmaf(A, offx, fmaf(B, offy2, C)) : 0.f;
            dst[3 + t] = make_float4(A, B, Cp, Cp2);
            const float margin = (fabsf(Cp) + 8.f * (fabsf(A) + fabsf(B))) * 0x1p-20f + 0x1p-20f;
            const float mn = Cp + fminf(0.5f * A, 7.5f * A) + fminf(0.5f * B, ((float)ROWS - 0.5f) * B);
            pass = pass && !(mn > bound + margin);
        } else {
            // an unused slot: a line that is -inf everywhere adds 2^-inf = 0 to the sum and never
            // wins the maximum, so every record is evaluated with K lines
            const float ninf = -__int_as_float(0x7f800000);
            dst[3 + t] = make_float4(0.f, 0.f, ninf, ninf);
        }
    }
    dst[0] = make_float4(h0.z, bound, h0.w, __int_as_float(T));
    dst[1] = make_float4(h1.x, h1.y, h1.z, __uint_as_float(r));
    dst[2] = make_float4(offx, offy, 0.f, 0.f);
    return pass;
}

// Packed FP32 (add / sub / mul / fma .f32x2): one instruction does the arithmetic of two independent
// evaluations held in the two halves of a 64-bit register pair (the forward's two records of a
// pixel, the backward's two pixels of a lane), rounding each half exactly like the scalar
// instruction.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long x, y, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

// Terms of one (pixel, convex) pair kept for the backward.
struct PairTerms {
    float alpha, I, z, oI, phi2, S;
    float e[KMAX];
};

// returns 0 when the line pre-test rejects the pair, 1 when alpha < tau, 2 when it contributes;
// HALF selects the 8x4 origin (0 upper, 1 lower) the pixel's local coordinates refer to; NT = K,
// the scene's points per convex: every staged record carries K line slots (unused ones are -inf),
// so the line loops carry no per-line guards
template <int HALF, int NT>
__device__ __forceinline__ int eval_pair(const float4 *__restrict__ rec, float lx, float ly, const Settings &st,
                                         PairTerms &p) {
    const float4 h0 = rec[0];
    float s[NT];
    float m = -__int_as_float(0x7f800000);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float4 L = rec[3 + t];
        s[t] = fmaf(L.x, lx, fmaf(L.y, ly, HALF ? L.w : L.z));
        m = fmaxf(m, s[t]);
    }
    if (m > h0.y) return 0;
    float S = 0.f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        p.e[t] = ex2(s[t] - m);
        S += p.e[t];
    }
    p.S = S;
    p.phi2 = m + lg2(S);
    p.z = ex2(h0.x * p.phi2);
    p.I = rcp(1.0f + p.z);
    p.oI = h0.z * p.I;
    p.alpha = fminf(st.alpha_max, p.oI);
    return p.alpha >= st.tau ? 2 : 1;
}

// work counters of the instrumented kernel variants: pairs visited, their hull lines, pairs past
// the line pre-test, their hull lines, contributing pairs, pixels
// eval_pair<0, NT> of two records for the same pixel at once, record 1 in the .x halves and record
// 2 in the .y halves of the packed arithmetic, with the same values and codes as two calls of
// eval_pair (two = false: record 2 is not evaluated and its code is 0).
template <int NT>
__device__ __forceinline__ void eval_two(const float4 *__restrict__ rec1, const float4 *__restrict__ rec2, bool two,
                                         float lx, float ly, const Settings &st, int &code1, int &code2,
                                         float2 &alpha) {
    const float4 h1 = rec1[0], h2 = rec2[0];
    float s1[NT], s2[NT];
    float m1 = -__int_as_float(0x7f800000), m2 = m1;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float4 L1 = rec1[3 + t], L2 = rec2[3 + t];
        s1[t] = fmaf(L1.x, lx, fmaf(L1.y, ly, L1.z));
        s2[t] = fmaf(L2.x, lx, fmaf(L2.y, ly, L2.z));
        m1 = fmaxf(m1, s1[t]);
        m2 = fmaxf(m2, s2[t]);
    }
    const bool act1 = !(m1 > h1.y), act2 = two && !(m2 > h2.y);
    code1 = code2 = 0;
    if (!(act1 || act2)) return;
    const float2 M = make_float2(m1, m2);
    float2 S = f2(0.f);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float2 d = sub2(make_float2(s1[t], s2[t]), M);
        S = add2(S, make_float2(ex2(d.x), ex2(d.y)));
    }
    const float2 phi2 = add2(M, make_float2(lg2(S.x), lg2(S.y)));
    const float2 zx = mul2(make_float2(h1.x, h2.x), phi2);
    const float2 zp = add2(f2(1.0f), make_float2(ex2(zx.x), ex2(zx.y)));
    const float2 oI = mul2(make_float2(h1.z, h2.z), make_float2(rcp(zp.x), rcp(zp.y)));
    alpha = make_float2(fminf(st.alpha_max, oI.x), fminf(st.alpha_max, oI.y));
    if (act1) code1 = alpha.x >= st.tau ? 2 : 1;
    if (act2) code2 = alpha.y >= st.tau ? 2 : 1;
}

constexpr int NCOUNT = 6;
__device__ __forceinline__ void flush_counts(unsigned long long *dst, const unsigned long long (&c)[NCOUNT]) {
#pragma unroll
    for (int q = 0; q < NCOUNT; ++q) {
        unsigned long long x = c[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(dst + q, x);
    }
}

__device__ __forceinline__ void count_pair(unsigned long long (&cnt)[NCOUNT], const float4 *rec, int code) {
    const unsigned T = (unsigned)__float_as_int(rec[0].w);
    cnt[0]++;
    cnt[1] += T;
    if (code) {
        cnt[2]++;
        cnt[3] += T;
    }
    if (code == 2) cnt[4]++;
}

__device__ __forceinline__ int find_view(const ViewDesc *__restrict__ views, int n_views, uint32_t g) {
    int v = 0;
    while (v + 1 < n_views && g >= views[v + 1].tile_base) ++v;
    return v;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Gathers, into slots sidx[0..nh), the pair indices of up to 32 records whose pixel box meets
// the warp's block [x0, x1] x [y0, y1] (pixel centres), scanning the tile's list from pos forwards
// (BACK = false, slots in increasing index order) or backwards from pos (BACK = true, slots in
// decreasing order), and advances pos past what it consumed.  Warp-uniform except the loads.
template <bool BACK>
__device__ __forceinline__ int gather_candidates(const BlendArgs &a, float x0, float x1, float y0, float y1,
                                                 uint32_t block_bits, uint32_t lo, uint32_t hi, uint32_t &pos,
                                                 uint32_t *sidx, int lane) {
    const uint32_t lt = lanemask_lt();
    int nh = 0;
    while (nh < 32 && (BACK ? pos > lo : pos < hi)) {
        const uint32_t avail = BACK ? pos - lo : hi - pos;
        const uint32_t i = BACK ? pos - 1 - (uint32_t)lane : pos + (uint32_t)lane;
        bool hit = false;
        if ((uint32_t)lane < avail) {
            if (a.mask_shift) {  // the pair key carries the box test of every 8x4 block of the tile
                hit = ((__ldg(a.pair_keys + i) >> a.mask_shift) & block_bits) != 0u;
            } else {
                const uint32_t r = a.pair_vals[i];
                if (checked(r < a.n_records, CS_BAD_RECORD)) {
                    const float4 bb = __ldg(a.bboxes + r);
                    hit = !(bb.z < x0 || bb.x > x1 || bb.w < y0 || bb.y > y1);
                }
            }
        }
        const uint32_t hits = __ballot_sync(0xffffffffu, hit);
        const int room = 32 - nh;
        uint32_t take = hits;
        uint32_t consumed = min(32u, avail);
        if (__popc(hits) > room) {  // keep the first `room` hits and resume after the last one kept
            take = 0;
            uint32_t h = hits;
            for (int k = 0; k < room; ++k) {
                take |= h & (0u - h);
                h &= h - 1;
            }
            consumed = 32u - (uint32_t)__clz(take);
        }
        if ((take >> lane) & 1u) sidx[nh + __popc(take & lt)] = i;
        nh += __popc(take);
        pos = BACK ? pos - consumed : pos + consumed;
    }
    __syncwarp();
    return nh;
}

__device__ __forceinline__ void tile_of(const ViewDesc &vd, uint32_t g, int &tx, int &ty) {
    const uint32_t local = g - vd.tile_base;
    tx = (int)(local % (uint32_t)vd.tiles_x);
    ty = (int)(local / (uint32_t)vd.tiles_x);
}

// per-lane state of the forward's pixel
struct FwdPixel {
    float T, C0, C1, C2;  // transmittance and colour so far
    uint32_t last;        // pair index + 1 of the last contributing pair (0: none)
    bool done;            // the pixel is outside the image, or its walk has ended
};

// Walks pairs [lo, hi) of a tile front to back for the warp's 8x4 block (origin ox, oy; this lane
// at (lx, ly) within it), compositing into each lane's pixel (Eq. 5 with the 3DGS cut-offs) until
// its transmittance falls below t_min.  Warp-uniform; lanes that are done take no part.
template <bool COUNT, int K>
__device__ __forceinline__ void walk_forward(const BlendArgs &a, uint32_t lo, uint32_t hi, int w, int lane, float ox,
                                             float oy, float lx, float ly, float4 *wrec, uint32_t *sidx, FwdPixel &q,
                                             unsigned long long (&cnt)[NCOUNT]) {
    const Settings &st = a.st;
    uint32_t pos = lo;
    while (pos < hi) {
        if (__all_sync(0xffffffffu, q.done)) break;
        // this warp's 8x4 block is column w & 1, row w >> 1 of the tile: mask bit w
        const int nh = gather_candidates<false>(a, ox + 0.5f, ox + 7.5f, oy + 0.5f, oy + 3.5f, 1u << w, lo, hi, pos,
                                                sidx, lane);
        const uint32_t rl = copy_records<K>(wrec, a.records, a.pair_vals, sidx, nh, lane, a.n_records);
        const bool pass = stage_record<4, K>(wrec, lane, nh, rl, ox, oy, st);
        __syncwarp();
        uint32_t bits = __ballot_sync(0xffffffffu, pass);
        if (!q.done) {
            // two records per iteration: their evaluations are independent (only the compositing
            // depends on the record in front), which doubles the work between dependent latencies
            while (bits) {
                const uint32_t j1 = (uint32_t)(__ffs(bits) - 1);
                bits &= bits - 1;
                const uint32_t j2 = bits ? (uint32_t)(__ffs(bits) - 1) : j1;
                const bool two = bits != 0;
                bits &= bits - 1;
                const float4 *rec1 = wrec + j1 * SREC<K>, *rec2 = wrec + j2 * SREC<K>;
                int code1, code2;
                float2 al;
                eval_two<K>(rec1, rec2, two, lx, ly, st, code1, code2, al);
                if (COUNT) {
                    count_pair(cnt, rec1, code1);
                    if (two) count_pair(cnt, rec2, code2);
                }
                if (code1 == 2) {
                    const float4 c = rec1[1];
                    const float wgt = al.x * q.T;
                    q.C0 = fmaf(wgt, c.x, q.C0);
                    q.C1 = fmaf(wgt, c.y, q.C1);
                    q.C2 = fmaf(wgt, c.z, q.C2);
                    q.T = q.T * (1.0f - al.x);
                    q.last = sidx[j1] + 1;
                    if (q.T < st.t_min) {
                        q.done = true;
                        break;
                    }
                }
                if (code2 == 2) {
                    const float4 c = rec2[1];
                    const float wgt = al.y * q.T;
                    q.C0 = fmaf(wgt, c.x, q.C0);
                    q.C1 = fmaf(wgt, c.y, q.C1);
                    q.C2 = fmaf(wgt, c.z, q.C2);
                    q.T = q.T * (1.0f - al.y);
                    q.last = sidx[j2] + 1;
                    if (q.T < st.t_min) {
                        q.done = true;
                        break;
                    }
                }
            }
        }
        __syncwarp();
    }
}

// Tile split (tile_split = N > 0).  A tile with more than N pairs is heavy: its list is cut into
// chunks of N pairs, blended by separate CTAs (MODE_CHUNK) from T = 1 into a per-pixel chunk
// state, then merged by one CTA per heavy tile (MODE_MERGE) in depth order:
//     C = C_a + T_a C_b,  T = T_a T_b
// A chunk's own walk stops once its local transmittance falls below t_min, which is safe (the
// global transmittance is at most the local one).  Where T_a T_b < t_min the whole walk stops
// inside chunk b: the merge walks that chunk again from T_a for those pixels, so the cut-off is
// exactly the one of the unsplit walk.  The merge then leaves, for each chunk, the transmittance
// after it and the colour behind it (the backward's starting point for that chunk).
// Chunk state: [slot][5][256] floats, word 0-2 colour, 3 transmittance, 4 last pair + 1, for the
// tile pixel with index split_pixel(x, y) (x, y within the tile).
constexpr int MODE_PLAIN = 0, MODE_CHUNK = 1, MODE_MERGE = 2;
// MODE_PERSIST: one persistent launch over the tiles of several views (the batches of the serving
// loop): a grid of the CTAs resident at once, each taking the next tile of the order from a
// counter in device memory; the CTA that finishes a view's last tile raises the view's flag in
// mapped host memory, so that each view is known complete as soon as its image is written.
constexpr int MODE_PERSIST = 3;
constexpr int STATE_WORDS = 5;
constexpr uint32_t NO_SLOT = 0xffffffffu;

__device__ __forceinline__ int split_pixel(int x, int y) {
    return 32 * ((x >> 3) + 2 * (y >> 2)) + (x & 7) + 8 * (y & 3);  // the forward's thread of the pixel
}
__device__ __forceinline__ float *state_word(const BlendArgs &a, uint32_t slot, int word, int pix) {
    return a.chunk_state + ((size_t)slot * STATE_WORDS + word) * (TILE * TILE) + pix;
}

// the forward's outputs of pixel (px, py): colour over the background, final transmittance, last
// contributor
__device__ __forceinline__ void write_pixel(const ViewDesc &vd, const Settings &st, int px, int py, const FwdPixel &q) {
    const size_t hw = (size_t)vd.width * vd.height, pix = (size_t)py * vd.width + px;
    vd.image[pix] = fmaf(q.T, st.bg[0], q.C0);
    vd.image[hw + pix] = fmaf(q.T, st.bg[1], q.C1);
    vd.image[2 * hw + pix] = fmaf(q.T, st.bg[2], q.C2);
    if (vd.t_final) vd.t_final[pix] = q.T;
    vd.n_last[pix] = q.last;
}

// The whole forward of one 8x4 pixel block (column w & 1, row w >> 1 of tile g) by one warp: the
// walk over the tile's pairs and the outputs of the lane's pixel.
template <bool COUNT, int K>
__device__ __forceinline__ void forward_block(const BlendArgs &a, uint32_t g, int w, int lane, float4 *wrec,
                                              uint32_t *sidx, unsigned long long (&cnt)[NCOUNT]) {
    const ViewDesc &vd = a.views[find_view(a.views, a.n_views, g)];
    int tx, ty;
    tile_of(vd, g, tx, ty);
    const int bx = tx * TILE + (w & 1) * 8, by = ty * TILE + (w >> 1) * 4;
    const int px = bx + (lane & 7), py = by + (lane >> 3);
    const bool inside = px < vd.width && py < vd.height;
    const float lx = (float)(lane & 7) + 0.5f, ly = (float)(lane >> 3) + 0.5f;
    uint2 range = a.ranges[g];
    if (!checked(range.x <= range.y && range.y <= a.n_pairs, CS_BAD_RANGE)) range = make_uint2(0, 0);
    FwdPixel q{1.0f, 0.f, 0.f, 0.f, 0u, !inside};
    if (COUNT && inside) cnt[5]++;
    walk_forward<COUNT, K>(a, range.x, range.y, w, lane, (float)bx, (float)by, lx, ly, wrec, sidx, q, cnt);
    if (inside) write_pixel(vd, a.st, px, py, q);
}

template <bool COUNT, int K, int MODE>
__global__ void __launch_bounds__(FWD_THREADS, 4) k_blend_forward(BlendArgs a, unsigned long long *counts) {
    __shared__ float4 srec[FWD_THREADS / 32][STAGE_F4<K>];
    __shared__ uint32_t sidx_all[FWD_THREADS / 32][32];
    if (MODE == MODE_PERSIST) {
        __shared__ uint32_t s_item;
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        unsigned long long cnt[NCOUNT] = {0, 0, 0, 0, 0, 0};
        for (;;) {
            if (threadIdx.x == 0) s_item = atomicAdd(a.queue, 1u);
            __syncthreads();
            const uint32_t item = s_item;
            __syncthreads();  // every thread has the item before the next one is taken
            if (item >= a.n_tiles) break;
            const uint32_t g = a.tile_order[item];
            forward_block<false, K>(a, g, w, lane, srec[w], sidx_all[w], cnt);
            __threadfence();  // this thread's pixels, visible on the device before the count below
            __syncthreads();
            if (threadIdx.x == 0) {
                const int v = find_view(a.views, a.n_views, g);
                const uint32_t tiles = (uint32_t)(a.views[v].tiles_x * a.views[v].tiles_y);
                if (atomicAdd(a.view_tiles_done + v, 1u) + 1u == tiles) {  // the view's last tile
                    __threadfence_system();
                    *reinterpret_cast<volatile uint32_t *>(a.view_flags + v) = a.flag_value;
                }
            }
        }
        return;
    }
    uint32_t g, chunk = 0, slot = NO_SLOT;
    if (MODE == MODE_PLAIN) {
        g = a.tile_order ? a.tile_order[blockIdx.x] : a.tile_offset + blockIdx.x;
    } else {
        const uint2 it = (MODE == MODE_CHUNK ? a.split_items : a.split_heavy)[blockIdx.x];
        g = it.x;
        if (MODE == MODE_CHUNK) {
            chunk = it.y;
            slot = a.split_slot[g];
        } else {
            slot = it.y;
        }
    }
    const ViewDesc &vd = a.views[find_view(a.views, a.n_views, g)];
    int tx, ty;
    tile_of(vd, g, tx, ty);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = tx * TILE + (w & 1) * 8, by = ty * TILE + (w >> 1) * 4;
    const int px = bx + (lane & 7), py = by + (lane >> 3);
    const bool inside = px < vd.width && py < vd.height;
    const float ox = (float)bx, oy = (float)by;
    const float lx = (float)(lane & 7) + 0.5f, ly = (float)(lane >> 3) + 0.5f;
    uint2 range = a.ranges[g];
    if (!checked(range.x <= range.y && range.y <= a.n_pairs, CS_BAD_RANGE)) range = make_uint2(0, 0);
    const Settings st = a.st;
    float4 *wrec = srec[w];
    uint32_t *sidx = sidx_all[w];

    FwdPixel q{1.0f, 0.f, 0.f, 0.f, 0u, !inside};
    unsigned long long cnt[NCOUNT] = {0, 0, 0, 0, 0, inside ? 1ull : 0ull};
    const int sp = threadIdx.x;  // == split_pixel of this thread's pixel
    if (MODE == MODE_MERGE) {
        const uint32_t nch = (range.y - range.x + a.split - 1) / a.split;
        // pass A, front to back over the chunks: the global state before each chunk (kept in word
        // 3 for pass B), and the chunk in which the walk stops, if any
        int stop = -1;
        float Cs0 = 0.f, Cs1 = 0.f, Cs2 = 0.f;  // colour before the stop chunk
        for (uint32_t c = 0; c < nch; ++c) {
            const float cc0 = *state_word(a, slot + c, 0, sp), cc1 = *state_word(a, slot + c, 1, sp);
            const float cc2 = *state_word(a, slot + c, 2, sp), tc = *state_word(a, slot + c, 3, sp);
            const uint32_t lc = __float_as_uint(*state_word(a, slot + c, 4, sp));
            *state_word(a, slot + c, 3, sp) = q.T;
            if (stop >= 0) continue;
            if (c == 0 || q.T * tc >= st.t_min) {  // chunk 0 starts at T = 1: its walk is the global one
                q.C0 = fmaf(q.T, cc0, q.C0);
                q.C1 = fmaf(q.T, cc1, q.C1);
                q.C2 = fmaf(q.T, cc2, q.C2);
                q.T *= tc;
                if (lc) q.last = lc;
                if (c == 0 && tc < st.t_min) stop = 0;
            } else {
                stop = (int)c;  // q holds the state before chunk c
                Cs0 = q.C0;
                Cs1 = q.C1;
                Cs2 = q.C2;
            }
        }
        if (!inside) stop = -1;
        // walk again, from the state before it, the chunk in which each pixel's walk stops
        for (uint32_t c = 1; c < nch; ++c) {
            if (!__any_sync(0xffffffffu, stop == (int)c)) continue;
            FwdPixel r = q;
            r.done = stop != (int)c;
            const uint32_t lo = range.x + c * a.split, hi = min(range.y, lo + a.split);
            walk_forward<false, K>(a, lo, hi, w, lane, ox, oy, lx, ly, wrec, sidx, r, cnt);
            if (stop == (int)c) q = r;
        }
        // pass B, back to front: per chunk the transmittance after it and the colour behind it
        float A0 = q.T * st.bg[0], A1 = q.T * st.bg[1], A2 = q.T * st.bg[2];
        float Tnext = q.T;
        for (int c = (int)nch - 1; c >= 0; --c) {
            const float cc0 = *state_word(a, slot + c, 0, sp), cc1 = *state_word(a, slot + c, 1, sp);
            const float cc2 = *state_word(a, slot + c, 2, sp), tb = *state_word(a, slot + c, 3, sp);
            const bool visited = stop < 0 || c <= stop;
            *state_word(a, slot + c, 0, sp) = visited ? A0 : q.T * st.bg[0];
            *state_word(a, slot + c, 1, sp) = visited ? A1 : q.T * st.bg[1];
            *state_word(a, slot + c, 2, sp) = visited ? A2 : q.T * st.bg[2];
            *state_word(a, slot + c, 3, sp) = visited ? Tnext : q.T;
            if (c == stop) {  // its contribution: what the walk added from the state before it
                A0 += q.C0 - Cs0;
                A1 += q.C1 - Cs1;
                A2 += q.C2 - Cs2;
            } else if (visited) {
                A0 = fmaf(tb, cc0, A0);
                A1 = fmaf(tb, cc1, A1);
                A2 = fmaf(tb, cc2, A2);
            }
            if (visited) Tnext = tb;
        }
    } else {
        uint32_t lo = range.x, hi = range.y;
        if (MODE == MODE_CHUNK && slot != NO_SLOT) {
            lo = range.x + chunk * a.split;
            hi = min(range.y, lo + a.split);
        }
        walk_forward<COUNT, K>(a, lo, hi, w, lane, ox, oy, lx, ly, wrec, sidx, q, cnt);
        if (MODE == MODE_CHUNK && slot != NO_SLOT) {
            *state_word(a, slot + chunk, 0, sp) = q.C0;
            *state_word(a, slot + chunk, 1, sp) = q.C1;
            *state_word(a, slot + chunk, 2, sp) = q.C2;
            *state_word(a, slot + chunk, 3, sp) = q.T;
            *state_word(a, slot + chunk, 4, sp) = __uint_as_float(q.last);
            return;
        }
    }
    if (inside) {
        const size_t hw = (size_t)vd.width * vd.height, pix = (size_t)py * vd.width + px;
        vd.image[pix] = fmaf(q.T, st.bg[0], q.C0);
        vd.image[hw + pix] = fmaf(q.T, st.bg[1], q.C1);
        vd.image[2 * hw + pix] = fmaf(q.T, st.bg[2], q.C2);
        if (vd.t_final) vd.t_final[pix] = q.T;
        vd.n_last[pix] = q.last;
    }
    if (COUNT) flush_counts(counts, cnt);
}

// The production forward (no tile split, no counters): CTAs of half a tile, 4 warps for the upper
// or lower 16x8 half of tile order[blockIdx.x / 2], 8 CTAs per SM.  A CTA's warps finish at
// different times and its slot is freed only when the last one is done; halving the CTA halves
// what a slow warp holds up (blend forward 0.310 -> 0.303 ms against whole-tile CTAs).
template <int K>
__global__ void __launch_bounds__(FWD_THREADS / 2, 8) k_blend_forward_half(BlendArgs a) {
    constexpr int WARPS = FWD_THREADS / 64;
    __shared__ float4 srec[WARPS][STAGE_F4<K>];
    __shared__ uint32_t sidx_all[WARPS][32];
    unsigned long long cnt[NCOUNT] = {0, 0, 0, 0, 0, 0};
    const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t g = a.tile_order ? a.tile_order[blockIdx.x >> 1] : a.tile_offset + (blockIdx.x >> 1);
    forward_block<false, K>(a, g, (int)(blockIdx.x & 1) * WARPS + wl, lane, srec[wl], sidx_all[wl], cnt);
}

// per-lane state of the backward's two pixels (rows r and r + 4 of the warp's 8x8 block)
struct BwdPixels {           // .x: the lane's upper pixel, .y: its lower pixel (4 rows down)
    float2 Tc;               // transmittance behind the pair being undone
    float2 G0, G1, G2;       // dL/dC
    float2 GS;               // dL/dC . (colour seen behind the current pair, times T)
    uint32_t last[2];        // pairs at or beyond this index did not contribute
};

// Per-pair gradient words of a lane, packed: 3t + 0 = sum g_t x, 3t + 1 = sum g_t y, 3t + 2 = sum
// g_t over the lane's two pixels (8x8-block coordinates), then dsigma', dopacity, dcolour (3); the
// array is padded to the warp reduction's group size (16, 24 or 32 words).
template <int NT>
struct PackedWords {
    static constexpr int SIG = 3 * NT, OPA = 3 * NT + 1, RGB = 3 * NT + 2, USED = 3 * NT + 5;
    static constexpr int N = USED <= 16 ? 16 : USED <= 24 ? 24 : 32;
    // gradient-record word of packed word l (l < USED)
    __device__ static __forceinline__ int dest(int l) { return l < SIG ? l : l + (G_SIG - SIG); }
};

// Undoes record rec (pair index idx, NT lines) for both pixels of the lane: recovers T in front
// of the pair, writes the lane's packed gradient words into v, and returns whether any of the two
// pixels received a contribution.  Per pixel, the operations and their rounding are those of the
// forward's evaluation (eval_pair), so alpha and T agree with the forward bit for bit.
template <int NT, bool COUNT>
__device__ __forceinline__ bool bwd_record(const float4 *__restrict__ rec, uint32_t idx, float2 LX, float2 LY,
                                           float lx, float ly, const Settings &st, BwdPixels &q,
                                           float (&v)[PackedWords<NT>::N], unsigned long long (&cnt)[NCOUNT]) {
    using PW = PackedWords<NT>;
    const float4 h0 = rec[0];
#pragma unroll
    for (int w = 0; w < PW::N; ++w) v[w] = 0.f;
    // line values of both pixels (the lower pixel's block origin is the record's second C)
    float2 s[NT];
    float m0 = -__int_as_float(0x7f800000), m1 = m0;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float4 L = rec[3 + t];
        s[t] = fma2(f2(L.x), LX, fma2(f2(L.y), LY, make_float2(L.z, L.w)));
        m0 = fmaxf(m0, s[t].x);
        m1 = fmaxf(m1, s[t].y);
    }
    const bool act0 = idx < q.last[0] && !(m0 > h0.y), act1 = idx < q.last[1] && !(m1 > h0.y);
    if (!(act0 || act1)) {
        if (COUNT) {
            if (idx < q.last[0]) count_pair(cnt, rec, 0);
            if (idx < q.last[1]) count_pair(cnt, rec, 0);
        }
        return false;
    }
    const float2 M = make_float2(m0, m1);
    float2 S = f2(0.f), e[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float2 d = sub2(s[t], M);
        e[t] = make_float2(ex2(d.x), ex2(d.y));
        S = add2(S, e[t]);
    }
    const float2 phi2 = add2(M, make_float2(lg2(S.x), lg2(S.y)));
    const float2 zx = mul2(f2(h0.x), phi2);
    const float2 z = make_float2(ex2(zx.x), ex2(zx.y));
    const float2 zp = add2(f2(1.0f), z);
    const float2 I = make_float2(rcp(zp.x), rcp(zp.y));
    const float2 oI = mul2(f2(h0.z), I);
    const float2 alpha = make_float2(fminf(st.alpha_max, oI.x), fminf(st.alpha_max, oI.y));
    const bool on0 = act0 && alpha.x >= st.tau, on1 = act1 && alpha.y >= st.tau;
    if (COUNT) {
        if (idx < q.last[0]) count_pair(cnt, rec, act0 ? (on0 ? 2 : 1) : 0);
        if (idx < q.last[1]) count_pair(cnt, rec, act1 ? (on1 ? 2 : 1) : 0);
    }
    if (!(on0 || on1)) return false;
    // both pixels are undone together; a pixel the pair does not reach keeps its state and adds
    // zeros (selected, never multiplied, so an infinite z there cannot leak a NaN)
    const float4 c = rec[1];
    const float2 om = sub2(f2(1.0f), alpha);  // 1 - alpha >= 1 - alpha_max > 0
    const float2 inv = make_float2(rcp(om.x), rcp(om.y));
    const float2 Tn = mul2(q.Tc, inv);  // transmittance in front of this pair
    // dC/dalpha = T_n c - S / (1 - alpha), S the colour behind: only dL/dC . S is needed
    const float2 Gc = fma2(q.G2, f2(c.z), fma2(q.G1, f2(c.y), mul2(q.G0, f2(c.x))));
    const float2 GSi = mul2(q.GS, inv);
    const float2 dalpha = fma2(Tn, Gc, make_float2(-GSi.x, -GSi.y));
    const float2 ta0 = mul2(Tn, alpha);
    const float2 ta = make_float2(on0 ? ta0.x : 0.f, on1 ? ta0.y : 0.f);
    const float2 pr = mul2(q.G0, ta), pg = mul2(q.G1, ta), pb = mul2(q.G2, ta);
    v[PW::RGB] = pr.x + pr.y;
    v[PW::RGB + 1] = pg.x + pg.y;
    v[PW::RGB + 2] = pb.x + pb.y;
    q.GS = fma2(ta, Gc, q.GS);
    q.Tc = make_float2(on0 ? Tn.x : q.Tc.x, on1 ? Tn.y : q.Tc.y);
    // alpha below the cap: opacity, sigma and line gradients
    const bool g0 = on0 && oI.x < st.alpha_max, g1 = on1 && oI.y < st.alpha_max;
    const float2 da = make_float2(g0 ? dalpha.x : 0.f, g1 ? dalpha.y : 0.f);
    const float2 po = mul2(da, I);
    v[PW::OPA] = po.x + po.y;
    const float2 dI = mul2(da, f2(h0.z));
    // I = 1/(1 + 2^x), dI/dx = -ln2 I (1 - I) = -ln2 z I^2
    const float2 dx0 = mul2(mul2(mul2(mul2(make_float2(-dI.x, -dI.y), f2(LN2)), z), I), I);
    const float2 dx = make_float2(g0 ? dx0.x : 0.f, g1 ? dx0.y : 0.f);
    const float2 ps = mul2(dx, phi2);
    v[PW::SIG] = ps.x + ps.y;
    const float2 dphi2 = mul2(mul2(dx, f2(h0.x)), make_float2(rcp(S.x), rcp(S.y)));
    // the two pixels share x; the lower one's y is 4 more
#pragma unroll
    for (int t = 0; t < NT; ++t) {
        const float2 gt = mul2(dphi2, e[t]);
        const float gs = gt.x + gt.y;
        v[3 * t] = gs * lx;
        v[3 * t + 1] = fmaf(gs, ly, 4.0f * gt.y);
        v[3 * t + 2] = gs;
    }
    return true;
}

// Reduce-scatter of N = 8, 16 or 32 values over the warp: returns, in lane l, the warp sum of
// v[l % N].  Recursive halving over lane bits log2(N) - 1 .. 0 (N - 1 shuffles), then a butterfly
// over the remaining lane bits (5 - log2(N) shuffles).
template <int N>
__device__ __forceinline__ float reduce_scatter(float (&v)[N], int lane) {
#pragma unroll
    for (int h = N / 2; h >= 1; h >>= 1) {
        const bool upper = (lane & h) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
            const float send = upper ? v[q] : v[q + h];
            const float keep = upper ? v[q + h] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    float x = v[0];
#pragma unroll
    for (int m = N; m < 32; m <<= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
    return x;
}

// lane l < USED receives the warp sum of packed word l
template <int N>
__device__ __forceinline__ float reduce_words(float (&v)[N], int lane) {
    if constexpr (N == 24) {
        float lo[16], hi[8];
#pragma unroll
        for (int w = 0; w < 16; ++w) lo[w] = v[w];
#pragma unroll
        for (int w = 0; w < 8; ++w) hi[w] = v[16 + w];
        const float a = reduce_scatter<16>(lo, lane);
        const float b = reduce_scatter<8>(hi, lane);
        return lane < 16 ? a : b;
    } else {
        return reduce_scatter<N>(v, lane);
    }
}

template <bool COUNT, int K, int MODE>
__global__ void __launch_bounds__(BWD_THREADS, 6) k_blend_backward(BlendArgs a, const float *__restrict__ dL_dimage,
                                                                int64_t image_stride, float4 *__restrict__ grads,
                                                                unsigned long long *counts) {
    __shared__ float4 srec[BWD_THREADS / 32][STAGE_F4<K>];
    __shared__ uint32_t sidx_all[BWD_THREADS / 32][32];
    uint32_t g, chunk = 0, slot = NO_SLOT;
    if (MODE == MODE_PLAIN) {
        g = a.tile_order ? a.tile_order[blockIdx.x] : a.tile_offset + blockIdx.x;
    } else {  // a chunk of a heavy tile (see the tile split of the forward), or a whole light tile
        const uint2 it = a.split_items[blockIdx.x];
        g = it.x;
        chunk = it.y;
        slot = a.split_slot[g];
    }
    const int v = find_view(a.views, a.n_views, g);
    const ViewDesc &vd = a.views[v];
    int tx, ty;
    tile_of(vd, g, tx, ty);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = tx * TILE + (w & 1) * 8, by = ty * TILE + (w >> 1) * 8;
    const float ox = (float)bx, oy = (float)by;
    const float lx = (float)(lane & 7) + 0.5f, ly = (float)(lane >> 3) + 0.5f;  // within each 8x4 half
    const int px = bx + (lane & 7);
    const Settings st = a.st;
    uint2 range = a.ranges[g];
    if (!checked(range.x <= range.y && range.y <= a.n_pairs, CS_BAD_RANGE)) range = make_uint2(0, 0);
    if (MODE == MODE_CHUNK && slot != NO_SLOT) {  // this chunk's pairs only
        range.x += chunk * a.split;
        range.y = min(range.y, range.x + a.split);
    }
    float4 *wrec = srec[w];
    uint32_t *sidx = sidx_all[w];

    // pixel k of this lane is row (lane >> 3) of the upper (k = 0) or lower (k = 1) 8x4 half
    BwdPixels q;
    float Tc[2], G0[2], G1[2], G2[2], GS[2];
    unsigned long long cnt[NCOUNT] = {0, 0, 0, 0, 0, 0};
    const size_t hw = (size_t)vd.width * vd.height;
    const float *dl = dL_dimage + v * image_stride;
    uint32_t lmax = 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int py = by + (lane >> 3) + 4 * k;
        Tc[k] = 1.0f;
        G0[k] = G1[k] = G2[k] = 0.f;
        q.last[k] = 0;
        if (px < vd.width && py < vd.height) {
            const size_t pix = (size_t)py * vd.width + px;
            G0[k] = dl[pix];
            G1[k] = dl[hw + pix];
            G2[k] = dl[2 * hw + pix];
            Tc[k] = vd.t_final[pix];
            q.last[k] = vd.n_last[pix];
            cnt[5]++;
        }
        // colour seen behind the current pair (T_after times its colour, summed from the back),
        // kept as its product with dL/dC; it starts with the background
        GS[k] = Tc[k] * fmaf(G2[k], st.bg[2], fmaf(G1[k], st.bg[1], G0[k] * st.bg[0]));
        if (MODE == MODE_CHUNK && slot != NO_SLOT) {
            // a chunk of a heavy tile starts from the transmittance after it and the colour behind
            // it, left by the forward's merge; its walk covers its own pairs only
            const int spx = split_pixel(bx - tx * TILE + (lane & 7), by - ty * TILE + (lane >> 3) + 4 * k);
            Tc[k] = *state_word(a, slot + chunk, 3, spx);
            GS[k] = fmaf(G2[k], *state_word(a, slot + chunk, 2, spx),
                         fmaf(G1[k], *state_word(a, slot + chunk, 1, spx), G0[k] * *state_word(a, slot + chunk, 0, spx)));
            q.last[k] = min(q.last[k], range.y);
        }
        lmax = max(lmax, q.last[k]);
    }
    q.Tc = make_float2(Tc[0], Tc[1]);
    q.G0 = make_float2(G0[0], G0[1]);
    q.G1 = make_float2(G1[0], G1[1]);
    q.G2 = make_float2(G2[0], G2[1]);
    q.GS = make_float2(GS[0], GS[1]);
    const float2 LX = f2(lx), LY = f2(ly);
    const uint32_t wend = __reduce_max_sync(0xffffffffu, lmax);
    uint32_t pos = max(wend, range.x);
    while (pos > range.x) {
        // this warp's 8x8 block is the 8x4 blocks of column w & 1, rows 2 (w >> 1) and 2 (w >> 1) + 1
        const uint32_t bbits = 5u << (4 * (w >> 1) + (w & 1));
        const int nh = gather_candidates<true>(a, ox + 0.5f, ox + 7.5f, oy + 0.5f, oy + 7.5f, bbits, range.x, range.y,
                                               pos, sidx, lane);
        bool pass = false;
        if (lane < nh) {
            uint32_t r = a.pair_vals[sidx[lane]];
            if (!checked(r < a.n_records, CS_BAD_RECORD)) r = 0;
            pass = stage_record_ldg<8, K>(wrec + lane * SREC<K>, a.records, r, ox, oy, st);
        }
        __syncwarp();
        uint32_t bits = __ballot_sync(0xffffffffu, pass);
        while (bits) {  // warp-uniform; slots hold decreasing pair indices
            const int j = __ffs(bits) - 1;
            bits &= bits - 1;
            const float4 *rec = wrec + j * SREC<K>;
            const uint32_t idx = sidx[j];
            using PW = PackedWords<K>;
            float v[PW::N];
            const bool any_on = bwd_record<K, COUNT>(rec, idx, LX, LY, lx, ly, st, q, v, cnt);
            if (!__any_sync(0xffffffffu, any_on)) continue;
            // lane l < PW::USED: the warp sum of packed word l
            float word = reduce_words<PW::N>(v, lane);
            // s = A (x8 + ox - ax) + B (y8 + oy - ay) + C: dA = sum(g x8) + (ox - ax) sum(g), dB likewise
            const float g2 = __shfl_down_sync(0xffffffffu, word, 2);
            const float g1 = __shfl_down_sync(0xffffffffu, word, 1);
            const uint32_t r = __float_as_uint(rec[1].w);
            if (lane < PW::SIG) {
                const int slot = lane % 3;
                if (slot == 0) word = fmaf(rec[2].x, g2, word);
                else if (slot == 1) word = fmaf(rec[2].y, g1, word);
            }
            if (lane < PW::USED && word != 0.f)
                atomicAdd(reinterpret_cast<float *>(grads + (size_t)r * (GRAD_WORDS / 4)) + PW::dest(lane), word);
        }
        __syncwarp();
    }
    if (COUNT) flush_counts(counts, cnt);
}

// launch order: class of a tile = 31 - floor(log2(pairs + 1)), longest lists in the first class
__device__ __forceinline__ uint32_t order_class(const uint2 &r) {
    const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
    return (uint32_t)__clz(len + 1u);  // 31 for an empty tile, smaller for longer lists
}
// the class of tile g in the view-by-view order: its view's classes come after those of the views
// before it
__device__ __forceinline__ uint32_t order_class_by_view(const uint2 *ranges, const ViewDesc *views, int n_views,
                                                        uint32_t g) {
    return (uint32_t)find_view(views, n_views, g) * TILE_ORDER_CLASSES + order_class(ranges[g]);
}

// One CTA: a histogram of the classes, their exclusive scan, then each tile placed at the next free
// slot of its class.  Lanes of a warp that share a class take their slots with one shared atomic.
constexpr int ORDER_THREADS = 1024, ORDER_PER = 8;

__device__ __forceinline__ uint32_t order_slot(uint32_t *counter, uint32_t c, bool active) {
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (!active) return 0;
    const unsigned peers = __match_any_sync(act, c);
    const int lead = __ffs(peers) - 1;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == lead) base = atomicAdd(&counter[c], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, lead);
    return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

constexpr int ORDER_CLASSES_MAX = TILE_ORDER_CLASSES * MAX_ORDER_VIEWS;
static_assert(ORDER_CLASSES_MAX == ORDER_THREADS, "one class per thread in the scan");

__global__ void __launch_bounds__(ORDER_THREADS) k_tile_order(const uint2 *__restrict__ ranges, uint32_t n_tiles,
                                                            uint32_t *__restrict__ order,
                                                            const ViewDesc *__restrict__ views, int n_views,
                                                            bool by_view, uint32_t *zero_words, int n_zero) {
    __shared__ uint32_t count[ORDER_CLASSES_MAX], next[ORDER_CLASSES_MAX], wsum[ORDER_THREADS / 32];
    const int n_classes = by_view ? TILE_ORDER_CLASSES * n_views : TILE_ORDER_CLASSES;
    count[threadIdx.x] = 0;
    for (int q = threadIdx.x; q < n_zero; q += ORDER_THREADS) zero_words[q] = 0u;
    __syncthreads();
    // ORDER_PER tiles per thread per round, their ranges loaded together (one load latency a round);
    // the bounds are the same for every lane of a warp, so the warp-wide votes see all 32 lanes
    const uint32_t stride = ORDER_THREADS * ORDER_PER;
    for (uint32_t base = 0; base < n_tiles; base += stride) {
        uint32_t c[ORDER_PER];
#pragma unroll
        for (int j = 0; j < ORDER_PER; ++j) {
            const uint32_t g = base + j * ORDER_THREADS + threadIdx.x;
            c[j] = g < n_tiles ? (by_view ? order_class_by_view(ranges, views, n_views, g) : order_class(ranges[g])) : 0u;
        }
#pragma unroll
        for (int j = 0; j < ORDER_PER; ++j) {
            const uint32_t g0 = base + j * ORDER_THREADS + (threadIdx.x & ~31u);
            if (g0 < n_tiles) order_slot(count, c[j], g0 + (threadIdx.x & 31u) < n_tiles);
        }
    }
    __syncthreads();
    {  // exclusive scan of the class sizes, one class per thread: within warps, then over them
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const uint32_t v = threadIdx.x < (unsigned)n_classes ? count[threadIdx.x] : 0u;
        uint32_t x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const uint32_t t = wsum[lane];
            uint32_t z = t;
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, z, d);
                if (lane >= d) z += y;
            }
            wsum[lane] = z - t;
        }
        __syncthreads();
        next[threadIdx.x] = wsum[wid] + x - v;
    }
    __syncthreads();
    for (uint32_t base = 0; base < n_tiles; base += stride) {
        uint32_t c[ORDER_PER];
#pragma unroll
        for (int j = 0; j < ORDER_PER; ++j) {
            const uint32_t g = base + j * ORDER_THREADS + threadIdx.x;
            c[j] = g < n_tiles ? (by_view ? order_class_by_view(ranges, views, n_views, g) : order_class(ranges[g])) : 0u;
        }
#pragma unroll
        for (int j = 0; j < ORDER_PER; ++j) {
            const uint32_t g0 = base + j * ORDER_THREADS + (threadIdx.x & ~31u);
            const uint32_t g = g0 + (threadIdx.x & 31u);
            if (g0 < n_tiles) {
                const uint32_t at = order_slot(next, c[j], g < n_tiles);
                if (g < n_tiles && checked(at < n_tiles, CS_BAD_TILE)) order[at] = g;
            }
        }
    }
}

// tile split planning: chunks of each heavy tile, 1 for each light tile
__global__ void k_split_count(const uint2 *__restrict__ ranges, uint32_t n_tiles, uint32_t split,
                              uint32_t *__restrict__ heavy, uint32_t *__restrict__ light,
                              unsigned int *__restrict__ n_heavy_tiles) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_tiles) return;
    const uint2 r = ranges[g];
    const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
    const uint32_t h = len > split ? (len + split - 1) / split : 0u;
    heavy[g] = h;
    light[g] = h ? 0u : 1u;
    const unsigned int nh = __reduce_add_sync(__activemask(), h ? 1u : 0u);
    if (nh && (threadIdx.x & 31) == __ffs(__activemask()) - 1) atomicAdd(n_heavy_tiles, nh);
}

__global__ void k_split_items(const uint2 *__restrict__ ranges, uint32_t n_tiles, uint32_t split,
                              const uint32_t *__restrict__ heavy_base, const uint32_t *__restrict__ light_base,
                              uint32_t n_slots, uint2 *__restrict__ items, uint2 *__restrict__ heavy_list,
                              unsigned int *__restrict__ heavy_fill, uint32_t *__restrict__ slot_of_tile) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_tiles) return;
    const uint2 r = ranges[g];
    const uint32_t len = r.y > r.x ? r.y - r.x : 0u;
    const uint32_t h = len > split ? (len + split - 1) / split : 0u;
    if (h) {
        const uint32_t base = heavy_base[g];
        for (uint32_t c = 0; c < h; ++c) items[base + c] = make_uint2(g, c);
        slot_of_tile[g] = base;
        heavy_list[atomicAdd(heavy_fill, 1u)] = make_uint2(g, base);
    } else {
        items[n_slots + light_base[g]] = make_uint2(g, 0u);
        slot_of_tile[g] = NO_SLOT;
    }
}

}  // namespace

// CTAs of a persistent launch: as many as are resident on the device at once (SMs x CTAs per SM
// at the kernel's occupancy), taken once per device; 0 when the query fails
template <typename F>
static uint32_t resident_ctas(F kernel, int threads, std::atomic<uint32_t> (&cache)[64]) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    uint32_t n = cache[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
            return 0;
        n = (uint32_t)(sms * per_sm);
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

template <int K>
static cudaError_t blend_forward_k(const BlendArgs &a, cudaStream_t s, unsigned long long *counts) {
    if (a.view_flags && !counts && !a.split) {
        static std::atomic<uint32_t> grid[64];
        const uint32_t n = min(a.n_tiles, resident_ctas(k_blend_forward<false, K, MODE_PERSIST>, FWD_THREADS, grid));
        if (n == 0) return cudaErrorInvalidConfiguration;
        k_blend_forward<false, K, MODE_PERSIST><<<n, FWD_THREADS, 0, s>>>(a, nullptr);
        return cudaSuccess;
    }
    if (counts) {
        k_blend_forward<true, K, MODE_PLAIN><<<a.n_tiles, FWD_THREADS, 0, s>>>(a, counts);
    } else if (a.split) {
        if (a.n_items) k_blend_forward<false, K, MODE_CHUNK><<<a.n_items, FWD_THREADS, 0, s>>>(a, nullptr);
        if (a.n_heavy) k_blend_forward<false, K, MODE_MERGE><<<a.n_heavy, FWD_THREADS, 0, s>>>(a, nullptr);
    } else {
        k_blend_forward_half<K><<<2 * a.n_tiles, FWD_THREADS / 2, 0, s>>>(a);
    }
    return cudaSuccess;
}

cudaError_t launch_blend_forward(const BlendArgs &a, cudaStream_t s, unsigned long long *counts) {
    if (a.n_tiles == 0) return cudaSuccess;
    cudaError_t e;
    switch (a.k) {
        case 3: e = blend_forward_k<3>(a, s, counts); break;
        case 4: e = blend_forward_k<4>(a, s, counts); break;
        case 5: e = blend_forward_k<5>(a, s, counts); break;
        case 6: e = blend_forward_k<6>(a, s, counts); break;
        case 7: e = blend_forward_k<7>(a, s, counts); break;
        case 8: e = blend_forward_k<8>(a, s, counts); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    count_launches(a.split && !counts ? (a.n_heavy ? 2 : 1) : 1);
    return cudaGetLastError();
}

template <int K>
static void blend_backward_k(const BlendArgs &a, const float *dL_dimage, int64_t image_stride, float4 *grad_records,
                             cudaStream_t s, unsigned long long *counts) {
    if (counts)
        k_blend_backward<true, K, MODE_PLAIN><<<a.n_tiles, BWD_THREADS, 0, s>>>(a, dL_dimage, image_stride, grad_records,
                                                                              counts);
    else if (a.split)
        k_blend_backward<false, K, MODE_CHUNK><<<a.n_items, BWD_THREADS, 0, s>>>(a, dL_dimage, image_stride,
                                                                               grad_records, nullptr);
    else
        k_blend_backward<false, K, MODE_PLAIN><<<a.n_tiles, BWD_THREADS, 0, s>>>(a, dL_dimage, image_stride,
                                                                               grad_records, nullptr);
}

cudaError_t take_status_blend(unsigned *bits, cudaStream_t s) {
#if CS_CHECKED
    unsigned v = 0;
    const unsigned zero = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_status_blend, sizeof v, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_status_blend, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) *bits |= v;
    return e;
#else
    (void)bits;
    (void)s;
    return cudaSuccess;
#endif
}

cudaError_t launch_tile_order(const uint2 *ranges, uint32_t n_tiles, uint32_t *order, const ViewDesc *views,
                              int n_views, bool by_view, uint32_t *zero_words, int n_zero, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    if (by_view && (n_views < 1 || n_views > MAX_ORDER_VIEWS)) return cudaErrorInvalidValue;
    k_tile_order<<<1, ORDER_THREADS, 0, s>>>(ranges, n_tiles, order, views, n_views, by_view, zero_words, n_zero);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_split_count(const uint2 *ranges, uint32_t n_tiles, uint32_t split, uint32_t *heavy, uint32_t *light,
                               unsigned int *n_heavy_tiles, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    k_split_count<<<(n_tiles + 255) / 256, 256, 0, s>>>(ranges, n_tiles, split, heavy, light, n_heavy_tiles);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_split_items(const uint2 *ranges, uint32_t n_tiles, uint32_t split, const uint32_t *heavy_base,
                               const uint32_t *light_base, uint32_t n_slots, uint2 *items, uint2 *heavy_list,
                               unsigned int *heavy_fill, uint32_t *slot_of_tile, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    k_split_items<<<(n_tiles + 255) / 256, 256, 0, s>>>(ranges, n_tiles, split, heavy_base, light_base, n_slots, items,
                                                        heavy_list, heavy_fill, slot_of_tile);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blend_backward(const BlendArgs &a, const float *dL_dimage, int64_t image_stride,
                                  float4 *grad_records, cudaStream_t s, unsigned long long *counts) {
    if (a.n_tiles == 0) return cudaSuccess;
    switch (a.k) {
        case 3: blend_backward_k<3>(a, dL_dimage, image_stride, grad_records, s, counts); break;
        case 4: blend_backward_k<4>(a, dL_dimage, image_stride, grad_records, s, counts); break;
        case 5: blend_backward_k<5>(a, dL_dimage, image_stride, grad_records, s, counts); break;
        case 6: blend_backward_k<6>(a, dL_dimage, image_stride, grad_records, s, counts); break;
        case 7: blend_backward_k<7>(a, dL_dimage, image_stride, grad_records, s, counts); break;
        case 8: blend_backward_k<8>(a, dL_dimage, image_stride, grad_records, s, counts); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace cs
