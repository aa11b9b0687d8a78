// Per-(view, convex) preprocess of the convex tile rasterizer, forward and backward.
//
// Forward (one thread per convex, points staged through shared memory with coalesced loads):
//   projection q_k = (fx x/z + cx, fy y/z + cy) of the K points            (Eq. 4)
//   centre c = mean p_k, camera distance d, scale d^p                       (Sec. 3.2, Eq. S1/S2)
//   exact-predicate Graham hull of the projected points                    (Sec. 3.2)
//   outward edge normals, conservative tile range, depth key               (Sec. 3.2, 2D Eq. 1)
//   lines pre-multiplied by log2(e) d^p delta, colour from SH              (Eq. S1, Sec. 3.2)
// The decisions (visibility, hull, tile range, depth key) are taken in IEEE binary32 with a fixed
// operation order and explicit round-to-nearest intrinsics, so they are reproducible bit for bit.
//
// Backward (one thread per drawn convex): chain rule from the per-record gradient accumulated by
// the blend backward to points, delta, sigma, opacity and SH.
#include "cs_common.cuh"

namespace cs {
namespace {

constexpr int PRE_THREADS = 128;
constexpr float COORD_LIMIT = 1048576.0f;  // 2^20 px
constexpr float LOG2E = 1.4426950408889634f;

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

// Natural logarithm in binary32 with a fixed operation order: x = m 2^e with m in [sqrt(1/2),
// sqrt(2)), ln m = 2 s (1 + s^2/3 + s^4/5 + ... + s^10/11), s = (m-1)/(m+1).  Used only for the
// tile-range radius, which must be identical wherever the range is computed.
__device__ float ln_series(float x) {
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

// Real spherical harmonics up to degree 3 at unit direction (x, y, z) and their gradients as
// polynomials on R^3.  Basis order l = 0..3, m = -l..l.
__device__ __forceinline__ void sh_eval(int deg, float x, float y, float z, float *Y, float (*dY)[3]) {
    const float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f;
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.5462742152960396f;
    const float C3a = 0.5900435899266435f, C3b = 2.890611442640554f, C3c = 0.4570457994644658f;
    const float C3d = 0.3731763325901154f, C3e = 1.445305721320277f;
    Y[0] = C0;
    if (dY) dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
    if (deg < 1) return;
    Y[1] = -C1 * y;
    Y[2] = C1 * z;
    Y[3] = -C1 * x;
    if (dY) {
        dY[1][0] = 0.f; dY[1][1] = -C1; dY[1][2] = 0.f;
        dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = C1;
        dY[3][0] = -C1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    }
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = C2a * x * y;
    Y[5] = -C2a * y * z;
    Y[6] = C2b * (2.f * zz - xx - yy);
    Y[7] = -C2a * x * z;
    Y[8] = C2c * (xx - yy);
    if (dY) {
        dY[4][0] = C2a * y; dY[4][1] = C2a * x; dY[4][2] = 0.f;
        dY[5][0] = 0.f; dY[5][1] = -C2a * z; dY[5][2] = -C2a * y;
        dY[6][0] = -2.f * C2b * x; dY[6][1] = -2.f * C2b * y; dY[6][2] = 4.f * C2b * z;
        dY[7][0] = -C2a * z; dY[7][1] = 0.f; dY[7][2] = -C2a * x;
        dY[8][0] = 2.f * C2c * x; dY[8][1] = -2.f * C2c * y; dY[8][2] = 0.f;
    }
    if (deg < 3) return;
    Y[9] = -C3a * y * (3.f * xx - yy);
    Y[10] = C3b * x * y * z;
    Y[11] = -C3c * y * (4.f * zz - xx - yy);
    Y[12] = C3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -C3c * x * (4.f * zz - xx - yy);
    Y[14] = C3e * z * (xx - yy);
    Y[15] = -C3a * x * (xx - 3.f * yy);
    if (dY) {
        dY[9][0] = -6.f * C3a * x * y; dY[9][1] = -3.f * C3a * (xx - yy); dY[9][2] = 0.f;
        dY[10][0] = C3b * y * z; dY[10][1] = C3b * x * z; dY[10][2] = C3b * x * y;
        dY[11][0] = 2.f * C3c * x * y; dY[11][1] = -C3c * (4.f * zz - xx - 3.f * yy); dY[11][2] = -8.f * C3c * y * z;
        dY[12][0] = -6.f * C3d * x * z; dY[12][1] = -6.f * C3d * y * z; dY[12][2] = C3d * (6.f * zz - 3.f * xx - 3.f * yy);
        dY[13][0] = -C3c * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * C3c * x * y; dY[13][2] = -8.f * C3c * x * z;
        dY[14][0] = 2.f * C3e * x * z; dY[14][1] = -2.f * C3e * y * z; dY[14][2] = C3e * (xx - yy);
        dY[15][0] = -3.f * C3a * (xx - yy); dY[15][1] = 6.f * C3a * x * y; dY[15][2] = 0.f;
    }
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

// colour = max(0, sum_j sh_j Y_j(dir) + 0.5) per channel; raw values (before the clamp) returned too
__device__ __forceinline__ void sh_colour(const float *__restrict__ sh, int deg, const float *Y, float raw[3]) {
    const int nb = (deg + 1) * (deg + 1);
    raw[0] = raw[1] = raw[2] = 0.5f;
    for (int j = 0; j < nb; ++j) {
        raw[0] += __ldg(sh + 3 * j + 0) * Y[j];
        raw[1] += __ldg(sh + 3 * j + 1) * Y[j];
        raw[2] += __ldg(sh + 3 * j + 2) * Y[j];
    }
}

template <int K>
__global__ void __launch_bounds__(PRE_THREADS) k_preprocess(const ViewDesc *__restrict__ views, Settings st,
                                                            PreprocessOut out) {
    const ViewDesc &vd = views[blockIdx.y];
    const int64_t n = vd.n;
    const int64_t i0 = (int64_t)blockIdx.x * PRE_THREADS;
    if (i0 >= n) return;
    __shared__ float sp[PRE_THREADS * K * 3];
    {
        const int64_t cnt = min((int64_t)PRE_THREADS, n - i0) * K * 3;
        const float *src = vd.points + i0 * K * 3;
        for (int j = threadIdx.x; j < cnt; j += PRE_THREADS) sp[j] = __ldg(src + j);
    }
    __syncthreads();
    const int64_t i = i0 + threadIdx.x;
    if (i >= n) return;
    const int64_t rec = vd.rec_base + i;
    const float *P = sp + threadIdx.x * K * 3;

    uint32_t depth_key = 0xffffffffu, count = 0;
    uint2 rect = make_uint2(0, 0);
    do {
        const float delta = __ldg(vd.delta + i), sigma = __ldg(vd.sigma + i), opa = __ldg(vd.opacity + i);
        bool finite = isfinite(delta) && isfinite(sigma) && isfinite(opa);
#pragma unroll
        for (int j = 0; j < 3 * K; ++j) finite = finite && isfinite(P[j]);
        if (!finite) break;
        if (!(delta > 0.f) || !(sigma > 0.f)) break;
        float u[K], v[K];
        bool ok = true;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float3 xc = xform(vd, P[3 * k], P[3 * k + 1], P[3 * k + 2]);
            ok = ok && (xc.z >= vd.z_near);
            u[k] = __fadd_rn(__fmul_rn(vd.fx, __fdiv_rn(xc.x, xc.z)), vd.cx);
            v[k] = __fadd_rn(__fmul_rn(vd.fy, __fdiv_rn(xc.y, xc.z)), vd.cy);
        }
        if (!ok) break;
#pragma unroll
        for (int k = 0; k < K; ++k) ok = ok && (fabsf(u[k]) <= COORD_LIMIT) && (fabsf(v[k]) <= COORD_LIMIT);
        if (!ok) break;
        // centre, distance, scale
        float c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float s = P[a];
#pragma unroll
            for (int k = 1; k < K; ++k) s = __fadd_rn(s, P[3 * k + a]);
            c[a] = __fdiv_rn(s, (float)K);
        }
        const float3 cc = xform(vd, c[0], c[1], c[2]);
        const float depth =
            __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(cc.x, cc.x), __fmul_rn(cc.y, cc.y)), __fmul_rn(cc.z, cc.z)));
        const float ds = st.dist_mode == 1 ? cc.z : depth;
        if (!(ds > 0.f) || !isfinite(ds) || !(depth > 0.f) || !isfinite(depth)) break;
        const float g = scale_power(ds, st.dist_power);
        const float dp = __fmul_rn(g, delta), spp = __fmul_rn(g, sigma);
        // opacity threshold
        float x = 0.f;
        bool full = false;
        if (st.tau > 0.f) {
            x = __fsub_rn(__fdiv_rn(opa, st.tau), 1.0f);
            if (!(x > 0.f)) break;
            if (!isfinite(x)) full = true;
        } else {
            if (!(opa > 0.f)) break;
            full = true;
        }
        // hull
        uint32_t hull;
        const int T = convex_hull<K>(u, v, hull);
        if (T < 3) break;
        float hu[KMAX], hv[KMAX], nx[KMAX], ny[KMAX];
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            if (t < T) {
                float a0, a1;
                select_point<K>(u, v, hull_pack_index(hull, t), a0, a1);
                hu[t] = a0;
                hv[t] = a1;
            }
        }
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            if (t >= T) break;
            const int t1 = (t + 1 == T) ? 0 : t + 1;
            float wx = hu[0], wy = hv[0];
#pragma unroll
            for (int q = 1; q < KMAX; ++q)
                if (q == t1) { wx = hu[q]; wy = hv[q]; }
            const float ex = __fsub_rn(wx, hu[t]), ey = __fsub_rn(wy, hv[t]);
            const float len = __fsqrt_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)));
            if (!(len > 0.f) || !isfinite(len)) { ok = false; }
            nx[t] = __fdiv_rn(ey, len);
            ny[t] = __fdiv_rn(-ex, len);
        }
        if (!ok) break;
        // conservative radius from phi >= d delta max_t L_t, then the mitre offset of the hull
        float r = 0.f;
        if (!full) {
            r = __fdiv_rn(ln_series(x), __fmul_rn(spp, dp));
            if (!isfinite(r)) full = true;
        }
        if (r < 0.f) r = 0.f;
        const float rp = __fadd_rn(__fmul_rn(r, 1.0009765625f), 0.00390625f);
        float xmin = 0.f, xmax = 0.f, ymin = 0.f, ymax = 0.f;
        if (!full) {
#pragma unroll
            for (int t = 0; t < KMAX; ++t) {
                if (t >= T) break;
                const int tp = (t == 0) ? T - 1 : t - 1;
                float pnx = nx[0], pny = ny[0];
#pragma unroll
                for (int q = 1; q < KMAX; ++q)
                    if (q == tp) { pnx = nx[q]; pny = ny[q]; }
                const float den = __fadd_rn(1.0f, __fadd_rn(__fmul_rn(pnx, nx[t]), __fmul_rn(pny, ny[t])));
                if (!(den > 0x1p-20f)) { full = true; break; }
                const float f = __fdiv_rn(rp, den);
                float ox = __fadd_rn(hu[t], __fmul_rn(f, __fadd_rn(pnx, nx[t])));
                float oy = __fadd_rn(hv[t], __fmul_rn(f, __fadd_rn(pny, ny[t])));
                ox = fminf(fmaxf(ox, -COORD_LIMIT), COORD_LIMIT);
                oy = fminf(fmaxf(oy, -COORD_LIMIT), COORD_LIMIT);
                if (t == 0) { xmin = xmax = ox; ymin = ymax = oy; }
                else {
                    xmin = fminf(xmin, ox); xmax = fmaxf(xmax, ox);
                    ymin = fminf(ymin, oy); ymax = fmaxf(ymax, oy);
                }
            }
        }
        int tx0, tx1, ty0, ty1;
        if (full) {
            tx0 = 0; ty0 = 0; tx1 = vd.tiles_x - 1; ty1 = vd.tiles_y - 1;
            xmin = ymin = -COORD_LIMIT;
            xmax = ymax = COORD_LIMIT;
        } else {
            tx0 = max((int)floorf(__fmul_rn(xmin, 0.0625f)), 0);
            tx1 = min((int)floorf(__fmul_rn(xmax, 0.0625f)), vd.tiles_x - 1);
            ty0 = max((int)floorf(__fmul_rn(ymin, 0.0625f)), 0);
            ty1 = min((int)floorf(__fmul_rn(ymax, 0.0625f)), vd.tiles_y - 1);
        }
        if (tx0 > tx1 || ty0 > ty1) break;

        // ---- continuous record (no bit-exactness needed beyond this point) ----
        const float kappa = dp * LOG2E;
        float w[REC_WORDS];
        w[R_AX] = hu[0];
        w[R_AY] = hv[0];
        w[R_SIG] = spp;
        w[R_OPA] = opa;
        {
            float Y[16];
            const float dx = c[0] - vd.campos[0], dy = c[1] - vd.campos[1], dz = c[2] - vd.campos[2];
            const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
            sh_eval(vd.sh_degree, dx * il, dy * il, dz * il, Y, nullptr);
            float raw[3];
            sh_colour(vd.sh + i * 3 * (vd.sh_degree + 1) * (vd.sh_degree + 1), vd.sh_degree, Y, raw);
            w[R_RGB + 0] = fmaxf(raw[0], 0.f);
            w[R_RGB + 1] = fmaxf(raw[1], 0.f);
            w[R_RGB + 2] = fmaxf(raw[2], 0.f);
        }
        w[R_HULL] = __uint_as_float(hull);
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            float A = 0.f, B = 0.f, C = 0.f;
            if (t < T) {
                A = kappa * nx[t];
                B = kappa * ny[t];
                C = kappa * (nx[t] * (hu[0] - hu[t]) + ny[t] * (hv[0] - hv[t]));
            }
            w[R_LINES + 3 * t] = A;
            w[R_LINES + 3 * t + 1] = B;
            w[R_LINES + 3 * t + 2] = C;
        }
        float4 *dst = out.records + rec * (REC_WORDS / 4);
#pragma unroll
        for (int q = 0; q < REC_WORDS / 4; ++q) dst[q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        out.bboxes[rec] = make_float4(xmin, ymin, xmax, ymax);
        depth_key = __float_as_uint(depth);
        count = (uint32_t)(tx1 - tx0 + 1) * (uint32_t)(ty1 - ty0 + 1);
        rect = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
    } while (false);
    out.depth_keys[rec] = depth_key;
    out.counts[rec] = count;
    out.rects[rec] = rect;
}

// ---------------------------------------------------------------------------------------------
// Backward preprocess
// ---------------------------------------------------------------------------------------------
// Backward: one thread per drawn convex.  With one view, the points and SH gradients of the
// block's convexes are accumulated (+=) in shared memory and read / written back with coalesced
// accesses; with several views, convexes are shared between views and use global atomics.
template <int K, int DEG, bool ATOMIC>
__global__ void __launch_bounds__(PRE_THREADS) k_preprocess_backward(const ViewDesc *__restrict__ views, Settings st,
                                                                     const float4 *__restrict__ records,
                                                                     const uint32_t *__restrict__ counts,
                                                                     const float4 *__restrict__ grads,
                                                                     PreprocessGrads out) {
    constexpr int NB = (DEG + 1) * (DEG + 1);
    constexpr int PW = K * 3, SW = NB * 3;           // words per convex
    constexpr int PS = PW | 1, SS = SW | 1;          // odd strides: no bank conflicts
    __shared__ float s_dp[ATOMIC ? 1 : PRE_THREADS * PS];
    __shared__ float s_dsh[ATOMIC ? 1 : PRE_THREADS * SS];
    const ViewDesc &vd = views[blockIdx.y];
    const int64_t i0 = (int64_t)blockIdx.x * PRE_THREADS;
    if (i0 >= vd.n) return;
    const int cnt = (int)min((int64_t)PRE_THREADS, vd.n - i0);
    if (!ATOMIC) {
        if (out.dpoints)
            for (int q = threadIdx.x; q < cnt * PW; q += PRE_THREADS) s_dp[(q / PW) * PS + q % PW] = out.dpoints[i0 * PW + q];
        if (out.dsh)
            for (int q = threadIdx.x; q < cnt * SW; q += PRE_THREADS) s_dsh[(q / SW) * SS + q % SW] = out.dsh[i0 * SW + q];
        __syncthreads();
    }
    const int64_t i = i0 + threadIdx.x;
    const int64_t rec = vd.rec_base + i;
    if (i < vd.n && counts[rec] != 0) {
        float gw[GRAD_WORDS];
        const float4 h0 = records[rec * (REC_WORDS / 4)], h1 = records[rec * (REC_WORDS / 4) + 1];
#pragma unroll
        for (int q = 0; q < GRAD_WORDS / 4; ++q) {
            const float4 b = grads[rec * (GRAD_WORDS / 4) + q];
            gw[4 * q] = b.x; gw[4 * q + 1] = b.y; gw[4 * q + 2] = b.z; gw[4 * q + 3] = b.w;
        }
        (void)h0;
        const uint32_t hull = __float_as_uint(h1.w);
        const int T = (int)hull_pack_count(hull);
        const float *P = vd.points + i * PW;
        const float delta = vd.delta[i], sigma = vd.sigma[i];
        float p[K][3], xc[K][3], u[K], v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            p[k][0] = P[3 * k];
            p[k][1] = P[3 * k + 1];
            p[k][2] = P[3 * k + 2];
            const float3 x = xform(vd, p[k][0], p[k][1], p[k][2]);
            xc[k][0] = x.x; xc[k][1] = x.y; xc[k][2] = x.z;
            u[k] = __fadd_rn(__fmul_rn(vd.fx, __fdiv_rn(x.x, x.z)), vd.cx);
            v[k] = __fadd_rn(__fmul_rn(vd.fy, __fdiv_rn(x.y, x.z)), vd.cy);
        }
        float c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float sum = p[0][a];
#pragma unroll
            for (int k = 1; k < K; ++k) sum = __fadd_rn(sum, p[k][a]);
            c[a] = __fdiv_rn(sum, (float)K);
        }
        const float3 cc = xform(vd, c[0], c[1], c[2]);
        const float depth = sqrtf(cc.x * cc.x + cc.y * cc.y + cc.z * cc.z);
        const float ds = st.dist_mode == 1 ? cc.z : depth;
        const float g = scale_power(ds, st.dist_power);
        const float kappa = g * delta * LOG2E;

        // lines -> hull vertices -> projected points
        float hu[KMAX], hv[KMAX];
#pragma unroll
        for (int t = 0; t < KMAX; ++t)
            if (t < T) select_point<K>(u, v, hull_pack_index(hull, t), hu[t], hv[t]);
        const float ax = hu[0], ay = hv[0];
        float dkappa = 0.f;
        float dhu[KMAX], dhv[KMAX];
#pragma unroll
        for (int t = 0; t < KMAX; ++t) dhu[t] = dhv[t] = 0.f;
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            if (t >= T) break;
            const int t1 = (t + 1 == T) ? 0 : t + 1;
            float wx = hu[0], wy = hv[0];
#pragma unroll
            for (int q = 1; q < KMAX; ++q)
                if (q == t1) { wx = hu[q]; wy = hv[q]; }
            const float ex = wx - hu[t], ey = wy - hv[t];
            const float len = sqrtf(ex * ex + ey * ey);
            const float il = 1.0f / len;
            const float nx = ey * il, ny = -ex * il;
            const float gA = gw[3 * t], gB = gw[3 * t + 1], gC = gw[3 * t + 2];
            const float rx = ax - hu[t], ry = ay - hv[t];
            dkappa += gA * nx + gB * ny + gC * (nx * rx + ny * ry);
            const float dnx = kappa * (gA + gC * rx), dny = kappa * (gB + gC * ry);
            dhu[t] -= kappa * gC * nx;
            dhv[t] -= kappa * gC * ny;
            const float nd = nx * dnx + ny * dny;
            const float dux = (dnx - nx * nd) * il, duy = (dny - ny * nd) * il;
            const float dex = -duy, dey = dux;  // n = (ey, -ex)/|e|
#pragma unroll
            for (int q = 0; q < KMAX; ++q)
                if (q == t1) { dhu[q] += dex; dhv[q] += dey; }
            dhu[t] -= dex;
            dhv[t] -= dey;
        }
        float du[K], dv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) du[k] = dv[k] = 0.f;
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            if (t >= T) break;
            const int k = hull_pack_index(hull, t);
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (q == k) { du[q] += dhu[t]; dv[q] += dhv[t]; }
        }
        // delta, sigma, opacity, distance
        const float gsig = gw[G_SIG];
        const float dd_delta = dkappa * g * LOG2E, dd_sigma = gsig * g, dd_opa = gw[G_OPA];
        if (ATOMIC) {
            if (out.ddelta && dd_delta != 0.f) atomicAdd(out.ddelta + i, dd_delta);
            if (out.dsigma && dd_sigma != 0.f) atomicAdd(out.dsigma + i, dd_sigma);
            if (out.dopacity && dd_opa != 0.f) atomicAdd(out.dopacity + i, dd_opa);
        } else {
            if (out.ddelta) out.ddelta[i] += dd_delta;
            if (out.dsigma) out.dsigma[i] += dd_sigma;
            if (out.dopacity) out.dopacity[i] += dd_opa;
        }
        const float dg = dkappa * delta * LOG2E + gsig * sigma;
        float dds;
        if (st.dist_power == 1.0f) dds = dg;
        else if (st.dist_power == 0.0f) dds = 0.f;
        else if (st.dist_power == 0.5f) dds = dg * 0.5f / sqrtf(ds);
        else dds = dg * 2.f * ds;
        float dcc[3] = {0.f, 0.f, 0.f};
        if (st.dist_mode == 1) dcc[2] = dds;
        else { dcc[0] = dds * cc.x / depth; dcc[1] = dds * cc.y / depth; dcc[2] = dds * cc.z / depth; }
        float dc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) dc[a] = vd.R[a] * dcc[0] + vd.R[3 + a] * dcc[1] + vd.R[6 + a] * dcc[2];
        // colour: dsh and the gradient of the view direction (basis streamed term by term)
        {
            const float wx = c[0] - vd.campos[0], wy = c[1] - vd.campos[1], wz = c[2] - vd.campos[2];
            const float iwl = rsqrtf(wx * wx + wy * wy + wz * wz);
            const float dx = wx * iwl, dy = wy * iwl, dz = wz * iwl;
            const float *sh = vd.sh + i * SW;
            float raw0 = 0.5f, raw1 = 0.5f, raw2 = 0.5f;
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                float gx, gy, gz;
                const float Yj = sh_term(j, dx, dy, dz, gx, gy, gz);
                raw0 += __ldg(sh + 3 * j) * Yj;
                raw1 += __ldg(sh + 3 * j + 1) * Yj;
                raw2 += __ldg(sh + 3 * j + 2) * Yj;
            }
            const float gr0 = raw0 > 0.f ? gw[G_RGB] : 0.f;
            const float gr1 = raw1 > 0.f ? gw[G_RGB + 1] : 0.f;
            const float gr2 = raw2 > 0.f ? gw[G_RGB + 2] : 0.f;
            float ddx = 0.f, ddy = 0.f, ddz = 0.f;
            if (gr0 != 0.f || gr1 != 0.f || gr2 != 0.f) {
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    float gx, gy, gz;
                    const float Yj = sh_term(j, dx, dy, dz, gx, gy, gz);
                    const float d0 = Yj * gr0, d1 = Yj * gr1, d2 = Yj * gr2;
                    if (ATOMIC) {
                        if (out.dsh) {
                            if (d0 != 0.f) atomicAdd(out.dsh + i * SW + 3 * j, d0);
                            if (d1 != 0.f) atomicAdd(out.dsh + i * SW + 3 * j + 1, d1);
                            if (d2 != 0.f) atomicAdd(out.dsh + i * SW + 3 * j + 2, d2);
                        }
                    } else {
                        s_dsh[threadIdx.x * SS + 3 * j] += d0;
                        s_dsh[threadIdx.x * SS + 3 * j + 1] += d1;
                        s_dsh[threadIdx.x * SS + 3 * j + 2] += d2;
                    }
                    if (DEG > 0) {
                        const float sg = __ldg(sh + 3 * j) * gr0 + __ldg(sh + 3 * j + 1) * gr1 + __ldg(sh + 3 * j + 2) * gr2;
                        ddx += sg * gx;
                        ddy += sg * gy;
                        ddz += sg * gz;
                    }
                }
            }
            const float dd = dx * ddx + dy * ddy + dz * ddz;
            dc[0] += (ddx - dx * dd) * iwl;
            dc[1] += (ddy - dy * dd) * iwl;
            dc[2] += (ddz - dz * dd) * iwl;
        }
        const float invK = 1.0f / (float)K;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float iz = 1.0f / xc[k][2];
            const float dx = du[k] * vd.fx * iz, dy = dv[k] * vd.fy * iz;
            const float dz = -(du[k] * vd.fx * xc[k][0] + dv[k] * vd.fy * xc[k][1]) * iz * iz;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float d = vd.R[a] * dx + vd.R[3 + a] * dy + vd.R[6 + a] * dz + dc[a] * invK;
                if (ATOMIC) {
                    if (out.dpoints && d != 0.f) atomicAdd(out.dpoints + i * PW + 3 * k + a, d);
                } else {
                    s_dp[threadIdx.x * PS + 3 * k + a] += d;
                }
            }
        }
    }
    if (!ATOMIC) {
        __syncthreads();
        if (out.dpoints)
            for (int q = threadIdx.x; q < cnt * PW; q += PRE_THREADS) out.dpoints[i0 * PW + q] = s_dp[(q / PW) * PS + q % PW];
        if (out.dsh)
            for (int q = threadIdx.x; q < cnt * SW; q += PRE_THREADS) out.dsh[i0 * SW + q] = s_dsh[(q / SW) * SS + q % SW];
    }
}

}  // namespace

cudaError_t launch_preprocess(const ViewDesc *views_dev, const ViewDesc *, int n_views, int64_t max_n, int k,
                              const Settings &st, const PreprocessOut &out, cudaStream_t s) {
    if (max_n <= 0 || n_views <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((max_n + PRE_THREADS - 1) / PRE_THREADS), (unsigned)n_views);
    switch (k) {
        case 3: k_preprocess<3><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out); break;
        case 4: k_preprocess<4><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out); break;
        case 5: k_preprocess<5><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out); break;
        case 6: k_preprocess<6><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out); break;
        case 7: k_preprocess<7><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out); break;
        case 8: k_preprocess<8><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

template <int K>
static void launch_pre_bwd_k(dim3 grid, cudaStream_t s, int deg, bool atomic, const ViewDesc *views_dev,
                             const Settings &st, const float4 *records, const uint32_t *counts, const float4 *grads,
                             const PreprocessGrads &g) {
#define CS_PRE_BWD(D, A) k_preprocess_backward<K, D, A><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, records, counts, grads, g)
    switch (deg * 2 + (atomic ? 1 : 0)) {
        case 0: CS_PRE_BWD(0, false); break;
        case 1: CS_PRE_BWD(0, true); break;
        case 2: CS_PRE_BWD(1, false); break;
        case 3: CS_PRE_BWD(1, true); break;
        case 4: CS_PRE_BWD(2, false); break;
        case 5: CS_PRE_BWD(2, true); break;
        case 6: CS_PRE_BWD(3, false); break;
        default: CS_PRE_BWD(3, true); break;
    }
#undef CS_PRE_BWD
}

cudaError_t launch_preprocess_backward(const ViewDesc *views_dev, int n_views, int64_t max_n, int k, int sh_degree,
                                       const Settings &st, const float4 *records, const uint32_t *counts,
                                       const float4 *grad_records, const PreprocessGrads &g, bool atomic,
                                       cudaStream_t s) {
    if (max_n <= 0 || n_views <= 0) return cudaSuccess;
    if (sh_degree < 0 || sh_degree > 3) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((max_n + PRE_THREADS - 1) / PRE_THREADS), (unsigned)n_views);
    switch (k) {
        case 3: launch_pre_bwd_k<3>(grid, s, sh_degree, atomic, views_dev, st, records, counts, grad_records, g); break;
        case 4: launch_pre_bwd_k<4>(grid, s, sh_degree, atomic, views_dev, st, records, counts, grad_records, g); break;
        case 5: launch_pre_bwd_k<5>(grid, s, sh_degree, atomic, views_dev, st, records, counts, grad_records, g); break;
        case 6: launch_pre_bwd_k<6>(grid, s, sh_degree, atomic, views_dev, st, records, counts, grad_records, g); break;
        case 7: launch_pre_bwd_k<7>(grid, s, sh_degree, atomic, views_dev, st, records, counts, grad_records, g); break;
        case 8: launch_pre_bwd_k<8>(grid, s, sh_degree, atomic, views_dev, st, records, counts, grad_records, g); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace cs
