// Device helpers shared by the forward and backward preprocess: exact orientation predicate and
// Graham hull, camera transform, distance power, real SH basis terms, typed parameter loads and
// asynchronous shared-memory staging.  Included by preprocess.cu and preprocess_backward.cu only.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cs_common.cuh"
#include "cs_spec_math.cuh"

namespace cs {
namespace {


constexpr int PRE_THREADS = 128;
constexpr float COORD_LIMIT = 1048576.0f;  // 2^20 px
constexpr float LOG2E = 1.4426950408889634f;

// Launch grid of the per-(view, convex) kernels: x = view (fastest), y and z = block of
// PRE_THREADS convexes (y below 65535, z counting the rows of y), so that the blocks of all views
// over the same convexes are scheduled together.
inline dim3 view_major_grid(int n_views, int64_t max_n) {
    const int64_t nblk = (max_n + PRE_THREADS - 1) / PRE_THREADS;
    const int64_t y = nblk < 65535 ? nblk : 65535;
    return dim3((unsigned)n_views, (unsigned)y, (unsigned)((nblk + y - 1) / y));
}

// ---------------------------------------------------------------------------------------------
// Exact orientation sign of three binary32 points: sign((b-a) x (c-a)).
// A binary32 evaluation with a forward error bound decides almost every case; the rest are
// decided exactly: every product of two binary32 numbers is exact in binary64, and the sign of a
// sum of binary64 numbers follows from a nonoverlapping expansion built with error-free additions
// (Shewchuk 1997, "Adaptive Precision Floating-Point Arithmetic and Fast Robust Geometric
// Predicates", Grow-Expansion).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = __dadd_rn(a, b);
    double bv = __dsub_rn(s, a);
    double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

__device__ __noinline__ int orient_exact(float ax, float ay, float bx, float by, float cx, float cy) {
    // (b-a) x (c-a) = bx cy - bx ay - ax cy - by cx + by ax + ay cx
    const double term[6] = {__dmul_rn((double)bx, (double)cy), -__dmul_rn((double)bx, (double)ay),
                            -__dmul_rn((double)ax, (double)cy), -__dmul_rn((double)by, (double)cx),
                            __dmul_rn((double)by, (double)ax), __dmul_rn((double)ay, (double)cx)};
    double h[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double q = term[i];
#pragma unroll
        for (int j = 0; j < i; ++j) {
            double s, e;
            two_sum(q, h[j], s, e);
            h[j] = e;
            q = s;
        }
        h[i] = q;
    }
#pragma unroll
    for (int i = 5; i >= 0; --i)
        if (h[i] != 0.0) return h[i] > 0.0 ? 1 : -1;
    return 0;
}

__device__ __forceinline__ int orient(float ax, float ay, float bx, float by, float cx, float cy) {
    const float l = __fmul_rn(__fsub_rn(bx, ax), __fsub_rn(cy, ay));
    const float r = __fmul_rn(__fsub_rn(by, ay), __fsub_rn(cx, ax));
    const float det = __fsub_rn(l, r);
    const float mag = __fadd_rn(fabsf(l), fabsf(r));
    // |det - exact| <= (3 eps + 16 eps^2) mag with eps = 2^-24 while nothing over- or underflows
    if (mag >= 0x1p-60f && mag <= 0x1p100f) {
        const float bound = mag * 0x1p-22f;
        if (det > bound) return 1;
        if (det < -bound) return -1;
    }
    return orient_exact(ax, ay, bx, by, cx, cy);
}

template <int K>
__device__ __forceinline__ void select_point(const float (&u)[K], const float (&v)[K], int i, float &x, float &y) {
    x = u[0];
    y = v[0];
#pragma unroll
    for (int j = 1; j < K; ++j)
        if (i == j) { x = u[j]; y = v[j]; }
}

// Canonical strictly convex hull of K <= 8 binary32 points: drop exact duplicates (keep the
// lowest index), pivot = least v then least u, the others ranked by polar angle about the pivot
// (collinear ones nearer first), then the Graham scan keeps strict left turns only.  Returns T
// and the packed vertex list (pivot first).
template <int K>
__device__ int convex_hull(const float (&u)[K], const float (&v)[K], uint32_t &packed) {
    uint32_t alive = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        bool dup = false;
#pragma unroll
        for (int j = 0; j < i; ++j) dup |= (u[j] == u[i]) && (v[j] == v[i]);
        if (!dup) alive |= 1u << i;
    }
    int p = 0;  // index 0 is never a duplicate
#pragma unroll
    for (int i = 1; i < K; ++i) {
        if (!(alive >> i & 1u)) continue;
        float pu, pv;
        select_point<K>(u, v, p, pu, pv);
        if (v[i] < pv || (v[i] == pv && u[i] < pu)) p = i;
    }
    float pu, pv;
    select_point<K>(u, v, p, pu, pv);
    const uint32_t cand = alive & ~(1u << p);
    int rank[K];
#pragma unroll
    for (int i = 0; i < K; ++i) rank[i] = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
        for (int j = i + 1; j < K; ++j) {
            if (!((cand >> i) & (cand >> j) & 1u)) continue;
            const int o = orient(pu, pv, u[i], v[i], u[j], v[j]);
            // i before j: j is at a larger angle, or on the same ray and farther away
            bool i_first;
            if (o != 0) i_first = o > 0;
            else if (v[i] != v[j]) i_first = v[i] < v[j];
            else i_first = u[i] < u[j];
            if (i_first) rank[j]++;
            else rank[i]++;
        }
    }
    uint32_t order = 0;
#pragma unroll
    for (int i = 0; i < K; ++i)
        if (cand >> i & 1u) order |= (uint32_t)i << (4 * rank[i]);
    const int nc = __popc(cand);
    uint32_t stack = (uint32_t)p;  // nibble s holds the s-th stack entry
    int ns = 1;
#pragma unroll
    for (int r = 0; r < K - 1; ++r) {
        if (r >= nc) break;
        const int c = (order >> (4 * r)) & 15;
        float cu, cv;
        select_point<K>(u, v, c, cu, cv);
        while (ns >= 2) {
            float au, av, bu, bv;
            select_point<K>(u, v, (stack >> (4 * (ns - 2))) & 15, au, av);
            select_point<K>(u, v, (stack >> (4 * (ns - 1))) & 15, bu, bv);
            if (orient(au, av, bu, bv, cu, cv) > 0) break;
            --ns;
        }
        stack = (stack & ~(15u << (4 * ns))) | ((uint32_t)c << (4 * ns));
        ++ns;
    }
    packed = (uint32_t)ns;
    for (int i = 0; i < ns; ++i) packed |= ((stack >> (4 * i)) & 7u) << (4 + 3 * i);
    return ns;
}

__device__ __forceinline__ float3 xform(const ViewDesc &vd, float px, float py, float pz) {
    float o[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        o[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(vd.R[3 * r], px), __fmul_rn(vd.R[3 * r + 1], py)),
                                   __fmul_rn(vd.R[3 * r + 2], pz)),
                         vd.t[r]);
    return make_float3(o[0], o[1], o[2]);
}

__device__ __forceinline__ float scale_power(float ds, float pw) {
    if (pw == 1.0f) return ds;
    if (pw == 0.0f) return 1.0f;
    if (pw == 0.5f) return __fsqrt_rn(ds);
    return __fmul_rn(ds, ds);  // 2 (other powers are rejected on the host)
}

// One real SH basis function Y_j and its gradient at (x, y, z); j is a constant after unrolling,
// so only that term's polynomial is evaluated (nothing is kept in arrays).
__device__ __forceinline__ float sh_term(int j, float x, float y, float z, float &gx, float &gy, float &gz) {
    const float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f;
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.5462742152960396f;
    const float C3a = 0.5900435899266435f, C3b = 2.890611442640554f, C3c = 0.4570457994644658f;
    const float C3d = 0.3731763325901154f, C3e = 1.445305721320277f;
    gx = gy = gz = 0.f;
    switch (j) {
        case 0: return C0;
        case 1: gy = -C1; return -C1 * y;
        case 2: gz = C1; return C1 * z;
        case 3: gx = -C1; return -C1 * x;
        case 4: gx = C2a * y; gy = C2a * x; return C2a * x * y;
        case 5: gy = -C2a * z; gz = -C2a * y; return -C2a * y * z;
        case 6: gx = -2.f * C2b * x; gy = -2.f * C2b * y; gz = 4.f * C2b * z; return C2b * (2.f * z * z - x * x - y * y);
        case 7: gx = -C2a * z; gz = -C2a * x; return -C2a * x * z;
        case 8: gx = 2.f * C2c * x; gy = -2.f * C2c * y; return C2c * (x * x - y * y);
        case 9: gx = -6.f * C3a * x * y; gy = -3.f * C3a * (x * x - y * y); return -C3a * y * (3.f * x * x - y * y);
        case 10: gx = C3b * y * z; gy = C3b * x * z; gz = C3b * x * y; return C3b * x * y * z;
        case 11:
            gx = 2.f * C3c * x * y; gy = -C3c * (4.f * z * z - x * x - 3.f * y * y); gz = -8.f * C3c * y * z;
            return -C3c * y * (4.f * z * z - x * x - y * y);
        case 12:
            gx = -6.f * C3d * x * z; gy = -6.f * C3d * y * z; gz = C3d * (6.f * z * z - 3.f * x * x - 3.f * y * y);
            return C3d * z * (2.f * z * z - 3.f * x * x - 3.f * y * y);
        case 13:
            gx = -C3c * (4.f * z * z - 3.f * x * x - y * y); gy = 2.f * C3c * x * y; gz = -8.f * C3c * x * z;
            return -C3c * x * (4.f * z * z - x * x - y * y);
        case 14: gx = 2.f * C3e * x * z; gy = -2.f * C3e * y * z; gz = C3e * (x * x - y * y); return C3e * z * (x * x - y * y);
        default: gx = -3.f * C3a * (x * x - y * y); gy = 6.f * C3a * x * y; return -C3a * x * (x * x - 3.f * y * y);
    }
}

// A parameter stored as STG (cs_storage), widened to binary32 (exactly, for the 16-bit types).
template <int STG>
__device__ __forceinline__ float ld_param(const void *p, int64_t i) {
    if (STG == CS_STORE_F16) return __half2float(__ldg(reinterpret_cast<const __half *>(p) + i));
    if (STG == CS_STORE_BF16) return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16 *>(p) + i));
    return __ldg(reinterpret_cast<const float *>(p) + i);
}

// element i of an STG array in shared memory, widened
template <int STG>
__device__ __forceinline__ float sm_param(const void *p, int i) {
    if (STG == CS_STORE_F32) return reinterpret_cast<const float *>(p)[i];
    const uint16_t b = reinterpret_cast<const uint16_t *>(p)[i];
    return STG == CS_STORE_F16 ? __half2float(__ushort_as_half(b)) : __uint_as_float((uint32_t)b << 16);
}

// Ampere-style asynchronous global -> shared copies (LDGSTS); completion is awaited with
// cp.async.wait_all, a wait on this thread's own copies that needs no polling loop.
__device__ __forceinline__ void cp_async_16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
// request the 128-byte line holding p into L2 (no register, no wait)
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.L2 [%0];" ::"l"(p)); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int SH_MAX_WORDS = 48;  // 3 x (3 + 1)^2

// ---- a block's SH coefficients staged in shared memory ----------------------------------------
// Convex t of the block starts at 16-byte chunk t * stride, the stride being its chunk count
// rounded up to an odd number, so that the 16-byte loads of 8 consecutive threads fall in 8
// distinct groups of 4 banks.  When a convex's coefficients are not a whole number of chunks
// (degrees 0 and 2) or the array is not 16-byte aligned, they are staged element by element at a
// stride of shw elements (stride 0 below), odd for degrees 0 and 2.
constexpr int SH_STAGE_WORDS = 52;  // 32-bit words per convex: 13 chunks (degree 3, binary32)

__host__ __device__ inline int sh_chunk_stride(int shw, int esz) {
    const int b = shw * esz;
    return (b % 16) ? 0 : ((b / 16) | 1);
}

// element e (a compile-time constant after unrolling) of a 16-byte chunk of STG values, widened
template <int STG>
__device__ __forceinline__ float chunk_elem(const uint4 &c, int e) {
    if (STG == CS_STORE_F32) return __uint_as_float(e == 0 ? c.x : e == 1 ? c.y : e == 2 ? c.z : c.w);
    const int q = e >> 1;
    const uint32_t u = q == 0 ? c.x : q == 1 ? c.y : q == 2 ? c.z : c.w;
    const uint16_t b = (e & 1) ? (uint16_t)(u >> 16) : (uint16_t)(u & 0xffffu);
    return STG == CS_STORE_F16 ? __half2float(__ushort_as_half(b)) : __uint_as_float((uint32_t)b << 16);
}

// Issues the asynchronous copy of the block's SH coefficients (cnt convexes from i0) into ssh
// (PRE_THREADS * SH_STAGE_WORDS words) and returns the layout's chunk stride (0: element layout).
// The caller waits with cp_async_wait_all() and a block barrier before reading.
template <int STG>
__device__ __forceinline__ int stage_sh(void *ssh, const void *sh, int64_t i0, int cnt, int shw) {
    constexpr int esz = STG == CS_STORE_F32 ? 4 : 2;
    const char *src = reinterpret_cast<const char *>(sh) + (size_t)i0 * shw * esz;
    char *dst = reinterpret_cast<char *>(ssh);
    const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    const int stride = aligned ? sh_chunk_stride(shw, esz) : 0;
    if (stride) {
        const int cpc = shw * esz / 16, n = cnt * cpc;
        for (int q = threadIdx.x; q < n; q += PRE_THREADS) {
            const int t = q / cpc;
            cp_async_16(dst + 16 * (t * stride + q - t * cpc), src + 16 * q);
        }
    } else {
        const int bytes = cnt * shw * esz;
        const int n16 = aligned ? bytes / 16 : 0;
        for (int q = threadIdx.x; q < n16; q += PRE_THREADS) cp_async_16(dst + 16 * q, src + 16 * q);
        if (STG == CS_STORE_F32) {
            for (int q = 4 * n16 + threadIdx.x; q < bytes / 4; q += PRE_THREADS) cp_async_4(dst + 4 * q, src + 4 * q);
        } else {  // 16-bit tail (or a 2-byte aligned array): plain copies, ordered by the caller's barrier
            const uint16_t *s16 = reinterpret_cast<const uint16_t *>(src);
            uint16_t *d16 = reinterpret_cast<uint16_t *>(dst);
            for (int q = 8 * n16 + threadIdx.x; q < bytes / 2; q += PRE_THREADS) d16[q] = __ldg(s16 + q);
        }
    }
    cp_async_commit();
    return stride;
}

// Raw colour 0.5 + sum_j c_j Y_j(d) of staged convex t (nb = (degree + 1)^2 basis functions),
// accumulated term by term in basis order.
template <int STG>
__device__ __forceinline__ void sh_colour(const void *ssh, int t, int shw, int stride, int nb, float dx, float dy,
                                          float dz, float raw[3]) {
    raw[0] = raw[1] = raw[2] = 0.5f;
    if (stride) {
        constexpr int EPC = STG == CS_STORE_F32 ? 4 : 8;  // elements per chunk
        const uint4 *s4 = reinterpret_cast<const uint4 *>(ssh) + t * stride;
        uint4 ch = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j < nb) {
                float gx, gy, gz;
                const float Yj = sh_term(j, dx, dy, dz, gx, gy, gz);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int w = 3 * j + c;
                    if (w % EPC == 0) ch = s4[w / EPC];
                    raw[c] += chunk_elem<STG>(ch, w % EPC) * Yj;
                }
            }
        }
    } else {
        const int sb = t * shw;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j < nb) {
                float gx, gy, gz;
                const float Yj = sh_term(j, dx, dy, dz, gx, gy, gz);
#pragma unroll
                for (int c = 0; c < 3; ++c) raw[c] += sm_param<STG>(ssh, sb + 3 * j + c) * Yj;
            }
        }
    }
}

}  // namespace
}  // namespace cs
