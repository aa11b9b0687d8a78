// Binary32 functions whose results decide discrete outcomes (tile ranges, refinement choices)
// and therefore have one fixed definition, mirrored operation by operation on the CPU side:
// every step is an explicitly rounded intrinsic, so no contraction or reordering can change a bit.
#pragma once

#include <cuda_runtime.h>

#include "cs_common.cuh"

namespace cs {

// Natural logarithm in binary32 with a fixed operation order: x = m 2^e with m in [sqrt(1/2),
// sqrt(2)), ln m = 2 s (1 + s^2/3 + s^4/5 + ... + s^10/11), s = (m-1)/(m+1).  Used for the
// tile-range radius and for the raw values of split children, which must be identical wherever
// they are computed.
__device__ __forceinline__ float ln_series(float x) {
    int e;
    float m = frexpf(x, &e);
    if (m < 0x1.6a09e6p-1f) {
        m = __fmul_rn(m, 2.0f);
        e = e - 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float p = 0x1.745d18p-4f;
    p = __fadd_rn(__fmul_rn(p, s2), 0x1.c71c72p-4f);
    p = __fadd_rn(__fmul_rn(p, s2), 0x1.24924ap-3f);
    p = __fadd_rn(__fmul_rn(p, s2), 0x1.99999ap-3f);
    p = __fadd_rn(__fmul_rn(p, s2), 0x1.555556p-2f);
    p = __fadd_rn(__fmul_rn(p, s2), 1.0f);
    const float lnm = __fmul_rn(__fmul_rn(2.0f, s), p);
    return __fadd_rn(__fmul_rn((float)e, 0x1.62e430p-1f), lnm);
}

// Parameter activations (Sec. 3.3): delta, sigma = exp(raw), o = sigmoid(raw).  The activated
// values decide the tile range, so exp has one fixed binary32 definition: x = k ln2 + r (Cody-Waite,
// ln2 as a 16-bit head, exact times any |k| < 256, plus a tail), |r| <= ln2/2, exp r by its Taylor
// polynomial of degree 7 in Horner form, times 2^k.  Below 2^-126 the result is 0, above the
// binary32 range +inf.  sigmoid(x) = 1/(1 + exp(-x)).
__device__ __forceinline__ float exp_act(float x) {
    if (x != x) return x;
    if (x > 88.72283935546875f) return __int_as_float(0x7f800000);
    if (x < -87.33654022216797f) return 0.0f;
    const float k = rintf(__fmul_rn(x, 0x1.715476p+0f));
    float r = __fsub_rn(x, __fmul_rn(k, 0x1.62e4p-1f));
    r = __fsub_rn(r, __fmul_rn(k, 0x1.7f7d1cp-20f));
    float p = 0x1.a01a02p-13f;
    p = __fadd_rn(__fmul_rn(p, r), 0x1.6c16c2p-10f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.111112p-7f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-5f);
    p = __fadd_rn(__fmul_rn(p, r), 0x1.555556p-3f);
    p = __fadd_rn(__fmul_rn(p, r), 0.5f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    p = __fadd_rn(__fmul_rn(p, r), 1.0f);
    const int ki = (int)k;
    if (ki > 127) return __fmul_rn(__fmul_rn(p, 0x1p127f), 2.0f);
    return __fmul_rn(p, __int_as_float((ki + 127) << 23));
}

__device__ __forceinline__ float sigmoid_act(float x) { return __fdiv_rn(1.0f, __fadd_rn(1.0f, exp_act(-x))); }

// Exact tile test (tighter binning).  The tile rectangle bounds the mitre-offset hull
// {q : max_t L_t(q) <= r}, which holds every pixel where o I >= tau.  A tile of the rectangle is
// kept unless one hull line's smallest value over the tile's pixel centres, a corner of
// [16 tx + 0.5, 16 tx + 15.5] x [16 ty + 0.5, 16 ty + 15.5] picked by the signs of the line's
// normal, exceeds r: that line then separates the tile from the set (a separating-axis test along
// the hull normals; the tile's own axes are the rectangle).  It runs on the lines as the screen
// record stores them (A, B, C per line, relative to the anchor (ax, ay), all scaled by kappa) against
// rk = kappa r, with a margin of 2^-20 times the magnitudes involved for binary32 rounding.
// Rectangles of SAT_MIN_TILES..SAT_MAX_TILES tiles that are not whole-screen are tested.
constexpr int SAT_MIN_TILES = 3;      // rectangles of 1 or 2 tiles are kept whole (nothing to gain)
constexpr int SAT_MAX_TILES = 1024;   // larger rectangles (and whole-screen ones) are kept whole
constexpr int SAT_SERIAL_TILES = 8;   // up to this size one thread tests a range; larger, its warp

__device__ __forceinline__ bool tile_kept(const float *lines, int T, float ax, float ay, float rk, int tx, int ty) {
    const float fx = (float)(16 * tx), fy = (float)(16 * ty);
    const float X0 = __fadd_rn(fx, 0.5f), X1 = __fadd_rn(fx, 15.5f);
    const float Y0 = __fadd_rn(fy, 0.5f), Y1 = __fadd_rn(fy, 15.5f);
    bool keep = true;
#pragma unroll
    for (int t = 0; t < KMAX; ++t) {
        if (t < T) {
            const float A = lines[3 * t], B = lines[3 * t + 1], C = lines[3 * t + 2];
            const float X = A >= 0.f ? X0 : X1, Y = B >= 0.f ? Y0 : Y1;
            const float pa = __fmul_rn(A, __fsub_rn(X, ax)), pb = __fmul_rn(B, __fsub_rn(Y, ay));
            const float L = __fadd_rn(__fadd_rn(pa, pb), C);
            const float mag = __fadd_rn(__fadd_rn(fabsf(pa), fabsf(pb)), fabsf(C));
            const float bound = __fadd_rn(rk, __fmul_rn(mag, 0x1p-20f));
            if (L > bound) keep = false;
        }
    }
    return keep;
}

}  // namespace cs
