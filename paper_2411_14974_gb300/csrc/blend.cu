// Per-tile blending of the convex tile rasterizer, forward and backward.
//
// One CTA of 256 threads per 16x16 tile; each warp owns an 8x4 pixel block, each thread one
// pixel.  The tile's depth-ordered convex records are staged in shared memory in batches (one
// record per thread, 128-byte coalesced gather), re-expressed relative to the tile origin so
// that every line is two FMAs per pixel.  Per pixel and convex (Eq. S1, S2 and 5):
//     s_t  = log2(e) d delta L_t(q)                     (T lines, 2 FMA each)
//     phi2 = max_t s_t + log2 sum_t 2^(s_t - max)       (= log2(e) phi)
//     I    = 1 / (1 + 2^(d sigma phi2))                 (= Sigmoid(-d sigma phi))
//     alpha = min(alpha_max, o I); skip if alpha < tau; C += T alpha c; T *= 1 - alpha
// A pair whose largest line value already forces alpha < tau is skipped without any
// transcendental (phi >= max_t s_t).  The whole CTA leaves a batch loop once every pixel's
// transmittance has dropped below t_min.
//
// The backward walks each tile's list in reverse from the last contributor of each pixel,
// recovering T before a pair as T_after / (1 - alpha), and accumulates d(loss)/d(record) per
// convex: the 29 per-pixel terms are summed across the warp by a reduce-scatter (31 shuffles,
// lane l ends with word l), across the warps of the tile in shared memory, and added to the
// convex's gradient record by one coalesced atomic instruction per (tile, record).  A staged record
// also carries an 8-bit mask of the warps whose 8x4 pixel block can pass the line pre-test at all;
// each warp iterates only the records of its ballot-built bit set.
#include "cs_common.cuh"

namespace cs {
namespace {

constexpr int BLEND_THREADS = 256;
constexpr int BATCH = 128;  // records staged per round
constexpr int SREC = 10;    // float4 per staged record
// staged record: [0] = (sigma', prefilter bound, o, T)   [1] = (r, g, b, -)
//                [2 + t] = (A_t, B_t, C_t relative to the tile origin, aux)
//                aux of line 0/1/2 = tile origin minus anchor (x, y), record index (backward)
// staged mask: bit w set when warp w may see alpha >= tau (warp-level cull)
constexpr float LN2 = 0.6931471805599453f;

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

__device__ __forceinline__ void stage_record(float4 *dst, uint32_t *mask_out, const float4 *__restrict__ records,
                                             uint32_t r, float tile_x0, float tile_y0, const Settings &st) {
    const float4 *src = records + (size_t)r * (REC_WORDS / 4);
    const float4 h0 = __ldg(src), h1 = __ldg(src + 1);
    const uint32_t hull = __float_as_uint(h1.w);
    const int T = (int)hull_pack_count(hull);
    float L[3 * KMAX];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        if (4 * q < 3 * T) {
            const float4 v = __ldg(src + 2 + q);
            L[4 * q] = v.x; L[4 * q + 1] = v.y; L[4 * q + 2] = v.z; L[4 * q + 3] = v.w;
        } else {
            L[4 * q] = L[4 * q + 1] = L[4 * q + 2] = L[4 * q + 3] = 0.f;
        }
    }
    const float offx = tile_x0 - h0.x, offy = tile_y0 - h0.y;
    // prefilter: alpha < tau whenever sigma' * max_t s_t > log2(o/tau - 1) (phi2 >= max_t s_t);
    // widened slightly so that it never rejects a pair the full evaluation keeps
    float bound = __int_as_float(0x7f800000);
    if (st.tau > 0.f) {
        const float x = h0.w / st.tau - 1.0f;
        if (isfinite(x)) {
            const float b = log2f(x) / h0.z;
            bound = b + fabsf(b) * 0x1p-10f + 0x1p-10f;
        }
    }
    // warp cull: warp w covers pixel centres lx in [8(w&1) + .5, 8(w&1) + 7.5], ly in
    // [4(w>>1) + .5, 4(w>>1) + 3.5]; if for some line the smallest value over that block exceeds
    // the bound (with a margin covering the per-pixel rounding), no pixel of the warp passes
    uint32_t wmask = 0xffu;
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        if (t < T) {
            const float A = L[3 * t], B = L[3 * t + 1], C = L[3 * t + 2];
            const float Cp = fmaf(A, offx, fmaf(B, offy, C));
            const float aux = t == 0 ? offx : (t == 1 ? offy : __uint_as_float(r));
            dst[2 + t] = make_float4(A, B, Cp, aux);
            const float margin = (fabsf(Cp) + 16.f * (fabsf(A) + fabsf(B))) * 0x1p-20f + 0x1p-20f;
#pragma unroll
            for (int w = 0; w < BLEND_THREADS / 32; ++w) {
                const float x0 = (float)((w & 1) * 8) + 0.5f, y0 = (float)((w >> 1) * 4) + 0.5f;
                const float mx = fminf(A * x0, A * (x0 + 7.f)), my = fminf(B * y0, B * (y0 + 3.f));
                if (Cp + mx + my > bound + margin) wmask &= ~(1u << w);
            }
        }
    }
    dst[0] = make_float4(h0.z, bound, h0.w, __int_as_float(T));
    dst[1] = make_float4(h1.x, h1.y, h1.z, 0.f);
    *mask_out = wmask;
}

// Records of the current batch that warp `wbit` has to evaluate, as a bit set over the batch
// (uniform across the warp): one ballot per 32 staged records.
__device__ __forceinline__ void warp_records(const uint32_t *smask, uint32_t nb, uint32_t wbit, int lane,
                                             uint32_t (&act)[BATCH / 32]) {
#pragma unroll
    for (int q = 0; q < BATCH / 32; ++q) {
        const uint32_t j = (uint32_t)(q * 32 + lane);
        act[q] = __ballot_sync(0xffffffffu, j < nb && (smask[j] & wbit));
    }
}

// Terms of one (pixel, convex) pair kept for the backward.
struct PairTerms {
    float alpha, I, z, oI, phi2, S;
    float e[KMAX];
};

// returns 0 when the line pre-test rejects the pair, 1 when alpha < tau, 2 when it contributes
__device__ __forceinline__ int eval_pair(const float4 *__restrict__ rec, float lx, float ly, const Settings &st,
                                         PairTerms &p) {
    const float4 h0 = rec[0];
    const int T = __float_as_int(h0.w);
    float s[KMAX];
    float m = -__int_as_float(0x7f800000);
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        if (t < T) {
            const float4 L = rec[2 + t];
            s[t] = fmaf(L.x, lx, fmaf(L.y, ly, L.z));
            m = fmaxf(m, s[t]);
        }
    }
    if (m > h0.y) return 0;
    float S = 0.f;
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        if (t < T) {
            p.e[t] = ex2(s[t] - m);
            S += p.e[t];
        }
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

__device__ __forceinline__ int find_view(const ViewDesc *__restrict__ views, int n_views, uint32_t g) {
    int v = 0;
    while (v + 1 < n_views && g >= views[v + 1].tile_base) ++v;
    return v;
}

__device__ __forceinline__ void pixel_of(int tid, int &lx, int &ly) {
    const int w = tid >> 5, lane = tid & 31;
    lx = (w & 1) * 8 + (lane & 7);
    ly = (w >> 1) * 4 + (lane >> 3);
}

template <bool COUNT>
__global__ void __launch_bounds__(BLEND_THREADS) k_blend_forward(BlendArgs a, unsigned long long *counts) {
    __shared__ float4 srec[BATCH * SREC];
    __shared__ uint32_t smask[BATCH];
    const uint32_t g = blockIdx.x;
    const ViewDesc &vd = a.views[find_view(a.views, a.n_views, g)];
    const uint32_t local = g - vd.tile_base;
    const int tx = (int)(local % (uint32_t)vd.tiles_x), ty = (int)(local / (uint32_t)vd.tiles_x);
    int lxi, lyi;
    pixel_of(threadIdx.x, lxi, lyi);
    const int px = tx * TILE + lxi, py = ty * TILE + lyi;
    const bool inside = px < vd.width && py < vd.height;
    const float lx = (float)lxi + 0.5f, ly = (float)lyi + 0.5f;
    const uint2 range = a.ranges[g];
    const Settings st = a.st;
    const int lane = threadIdx.x & 31;
    const uint32_t wbit = 1u << (threadIdx.x >> 5);

    float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    unsigned long long cnt[NCOUNT] = {0, 0, 0, 0, 0, inside ? 1ull : 0ull};
    for (uint32_t base = range.x; base < range.y; base += BATCH) {
        if (__syncthreads_and(done)) break;
        const uint32_t nb = min((uint32_t)BATCH, range.y - base);
        if (threadIdx.x < nb)
            stage_record(srec + threadIdx.x * SREC, smask + threadIdx.x, a.records, a.pair_vals[base + threadIdx.x],
                         (float)(tx * TILE), (float)(ty * TILE), st);
        __syncthreads();
        uint32_t act[BATCH / 32];
        warp_records(smask, nb, wbit, lane, act);
        if (done) continue;
#pragma unroll
        for (int q = 0; q < BATCH / 32; ++q) {
            uint32_t bits = act[q];
            while (bits) {
                const uint32_t j = (uint32_t)(q * 32 + __ffs(bits) - 1);
                bits &= bits - 1;
                PairTerms p;
                const float4 *rec = srec + j * SREC;
                const int code = eval_pair(rec, lx, ly, st, p);
                if (COUNT) {
                    const unsigned Tl = (unsigned)__float_as_int(rec[0].w);
                    cnt[0]++;
                    cnt[1] += Tl;
                    if (code) {
                        cnt[2]++;
                        cnt[3] += Tl;
                    }
                    if (code == 2) cnt[4]++;
                }
                if (code != 2) continue;
                const float4 c = rec[1];
                const float wgt = p.alpha * T;
                C0 = fmaf(wgt, c.x, C0);
                C1 = fmaf(wgt, c.y, C1);
                C2 = fmaf(wgt, c.z, C2);
                T = T * (1.0f - p.alpha);
                last = base + j + 1;
                if (T < st.t_min) {
                    done = true;
                    break;
                }
            }
            if (done) break;
        }
    }
    if (inside) {
        const size_t hw = (size_t)vd.width * vd.height, pix = (size_t)py * vd.width + px;
        vd.image[pix] = fmaf(T, st.bg[0], C0);
        vd.image[hw + pix] = fmaf(T, st.bg[1], C1);
        vd.image[2 * hw + pix] = fmaf(T, st.bg[2], C2);
        if (vd.t_final) vd.t_final[pix] = T;
        vd.n_last[pix] = last;
    }
    if (COUNT) flush_counts(counts, cnt);
}

template <bool COUNT>
__global__ void __launch_bounds__(BLEND_THREADS) k_blend_backward(BlendArgs a, const float *__restrict__ dL_dimage,
                                                                  int64_t image_stride, float4 *__restrict__ grads,
                                                                  unsigned long long *counts) {
    __shared__ float4 srec[BATCH * SREC];
    __shared__ uint32_t smask[BATCH];
    __shared__ float sgrad[BATCH * 32];  // per staged record: the gradient-record words of this tile
    __shared__ uint32_t s_max_last[BLEND_THREADS / 32];
    const uint32_t g = blockIdx.x;
    const int v = find_view(a.views, a.n_views, g);
    const ViewDesc &vd = a.views[v];
    const uint32_t local = g - vd.tile_base;
    const int tx = (int)(local % (uint32_t)vd.tiles_x), ty = (int)(local / (uint32_t)vd.tiles_x);
    int lxi, lyi;
    pixel_of(threadIdx.x, lxi, lyi);
    const int px = tx * TILE + lxi, py = ty * TILE + lyi;
    const bool inside = px < vd.width && py < vd.height;
    const float lx = (float)lxi + 0.5f, ly = (float)lyi + 0.5f;
    const uint2 range = a.ranges[g];
    const Settings st = a.st;
    const int lane = threadIdx.x & 31;

    float Tc = 1.0f, G0 = 0.f, G1 = 0.f, G2 = 0.f;
    uint32_t last = 0;
    if (inside) {
        const size_t hw = (size_t)vd.width * vd.height, pix = (size_t)py * vd.width + px;
        const float *dl = dL_dimage + v * image_stride;
        G0 = dl[pix];
        G1 = dl[hw + pix];
        G2 = dl[2 * hw + pix];
        Tc = vd.t_final[pix];
        last = vd.n_last[pix];
    }
    // colour seen behind the current pair, T_after * (its colour) summed from the back
    float S0 = Tc * st.bg[0], S1 = Tc * st.bg[1], S2 = Tc * st.bg[2];
    unsigned long long cnt[NCOUNT] = {0, 0, 0, 0, 0, inside ? 1ull : 0ull};
    uint32_t wl = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wl = max(wl, __shfl_xor_sync(0xffffffffu, wl, o));
    if (lane == 0) s_max_last[threadIdx.x >> 5] = wl;
    __syncthreads();
    uint32_t end = range.x;
#pragma unroll
    for (int q = 0; q < BLEND_THREADS / 32; ++q) end = max(end, s_max_last[q]);

    while (end > range.x) {
        const uint32_t start = end > range.x + BATCH ? end - BATCH : range.x;
        const uint32_t nb = end - start;
        __syncthreads();
        if (threadIdx.x < nb)
            stage_record(srec + threadIdx.x * SREC, smask + threadIdx.x, a.records, a.pair_vals[start + threadIdx.x],
                         (float)(tx * TILE), (float)(ty * TILE), st);
        for (uint32_t i = threadIdx.x; i < nb * 32; i += BLEND_THREADS) sgrad[i] = 0.f;
        __syncthreads();
        const uint32_t wbit = 1u << (threadIdx.x >> 5);
        uint32_t act[BATCH / 32];
        warp_records(smask, nb, wbit, lane, act);
#pragma unroll
        for (int q = BATCH / 32 - 1; q >= 0; --q) {
          uint32_t bits = act[q];
          while (bits) {  // warp-uniform, from the back of the batch
            const int jj = 31 - __clz(bits);
            bits &= ~(1u << jj);
            const int j = q * 32 + jj;
            const float4 *rec = srec + j * SREC;
            const uint32_t idx = start + (uint32_t)j;
            PairTerms p;
            const int code = idx < last ? eval_pair(rec, lx, ly, st, p) : -1;
            const bool on = code == 2;
            if (COUNT && code >= 0) {
                const unsigned T = (unsigned)__float_as_int(rec[0].w);
                cnt[0]++;
                cnt[1] += T;
                if (code) {
                    cnt[2]++;
                    cnt[3] += T;
                }
                if (on) cnt[4]++;
            }
            if (!__any_sync(0xffffffffu, on)) continue;
            const float4 h0 = rec[0];
            const int T = __float_as_int(h0.w);
            // per-pixel terms in gradient-record word order: 3t+0 = g_t lx, 3t+1 = g_t ly,
            // 3t+2 = g_t, 24 dsigma', 25 dopacity, 26..28 dcolour
            float v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = 0.f;
            if (on) {
                const float4 c = rec[1];
                const float om = 1.0f - p.alpha;
                const float inv = __frcp_rn(om);
                const float Tn = Tc * inv;  // transmittance in front of this pair
                const float dalpha = G0 * (Tn * c.x - S0 * inv) + G1 * (Tn * c.y - S1 * inv) + G2 * (Tn * c.z - S2 * inv);
                const float ta = Tn * p.alpha;
                v[G_RGB] = G0 * ta;
                v[G_RGB + 1] = G1 * ta;
                v[G_RGB + 2] = G2 * ta;
                S0 = fmaf(ta, c.x, S0);
                S1 = fmaf(ta, c.y, S1);
                S2 = fmaf(ta, c.z, S2);
                Tc = Tn;
                if (p.oI < st.alpha_max) {
                    v[G_OPA] = dalpha * p.I;
                    const float dI = dalpha * h0.z;
                    // I = 1/(1 + 2^x), dI/dx = -ln2 I (1 - I) = -ln2 z I^2
                    const float dx = -dI * LN2 * p.z * p.I * p.I;
                    v[G_SIG] = dx * p.phi2;
                    const float dphi2 = dx * h0.x * rcp(p.S);
#pragma unroll
                    for (int t = 0; t < KMAX; ++t) {
                        if (t < T) {
                            const float gt = dphi2 * p.e[t];
                            v[3 * t] = gt * lx;
                            v[3 * t + 1] = gt * ly;
                            v[3 * t + 2] = gt;
                        }
                    }
                }
            }
            // reduce-scatter across the warp: after five halvings lane l holds the warp sum of v[l]
#pragma unroll
            for (int h = 16; h >= 1; h >>= 1) {
                const bool upper = (lane & h) != 0;
#pragma unroll
                for (int q = 0; q < h; ++q) {
                    const float send = upper ? v[q] : v[q + h];
                    const float keep = upper ? v[q + h] : v[q];
                    v[q] = keep + __shfl_xor_sync(0xffffffffu, send, h);
                }
            }
            float word = v[0];
            // s = A (lx + offx) + B (ly + offy) + C: dA = sum(g lx) + offx sum(g), dB likewise
            const float g2 = __shfl_down_sync(0xffffffffu, word, 2);
            const float g1 = __shfl_down_sync(0xffffffffu, word, 1);
            const int slot = lane < 24 ? lane % 3 : 3;
            if (slot == 0) word = fmaf(rec[2].w, g2, word);
            else if (slot == 1) word = fmaf(rec[3].w, g1, word);
            if (lane < 29 && word != 0.f) atomicAdd(sgrad + j * 32 + lane, word);
          }
        }
        __syncthreads();
        // one coalesced global atomic per (tile, record, word) for what the warps accumulated
        for (uint32_t i = threadIdx.x; i < nb * 32; i += BLEND_THREADS) {
            const float w = sgrad[i];
            if (w != 0.f) {
                const uint32_t r = __float_as_uint(srec[(i >> 5) * SREC + 4].w);
                atomicAdd(reinterpret_cast<float *>(grads + (size_t)r * (GRAD_WORDS / 4)) + (i & 31), w);
            }
        }
        end = start;
    }
    if (COUNT) flush_counts(counts, cnt);
}

}  // namespace

cudaError_t launch_blend_forward(const BlendArgs &a, cudaStream_t s, unsigned long long *counts) {
    if (a.n_tiles == 0) return cudaSuccess;
    if (counts) k_blend_forward<true><<<a.n_tiles, BLEND_THREADS, 0, s>>>(a, counts);
    else k_blend_forward<false><<<a.n_tiles, BLEND_THREADS, 0, s>>>(a, nullptr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blend_backward(const BlendArgs &a, const float *dL_dimage, int64_t image_stride,
                                  float4 *grad_records, cudaStream_t s, unsigned long long *counts) {
    if (a.n_tiles == 0) return cudaSuccess;
    if (counts)
        k_blend_backward<true><<<a.n_tiles, BLEND_THREADS, 0, s>>>(a, dL_dimage, image_stride, grad_records, counts);
    else
        k_blend_backward<false><<<a.n_tiles, BLEND_THREADS, 0, s>>>(a, dL_dimage, image_stride, grad_records, nullptr);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace cs
