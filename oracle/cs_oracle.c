/*
 * CPU oracle for the differentiable tile rasterizer of 3D Convex Splatting (arXiv 2411.14974).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference against which the CUDA path
 * is checked; the product never links, loads or calls it.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may use it.  It shares no code, header or constant
 * generator with the CUDA sources.
 *
 * Two parts:
 *
 *  (1) Discrete specification, evaluated in IEEE binary32 with a fixed operation order and no
 *      contraction (build with -ffp-contract=off).  It decides, per convex, whether it is drawn,
 *      the 2D convex hull (Sec. 3.2, "2D convex hull computation"; Graham scan with exact
 *      orientation predicates), the conservative screen rectangle of tiles it may touch, and the
 *      sort key "distance from the camera to the centre" (Sec. 3.2, before Eq. 5).  These are the
 *      integer decisions the GPU has to reproduce bit for bit, so both sides take them in float32.
 *
 *  (2) Continuous render in binary64, brute force over every convex for every requested pixel,
 *      no tiles: projection (Eq. 4, with the perspective divide), hull lines (2D form of Eq. 1),
 *      smooth indicator with distance scaling (Eq. S1/S2 of the supplement, i.e. Eq. 2/3 in 2D),
 *      spherical-harmonic colour, and front-to-back alpha compositing (Eq. 5).  The analytic
 *      binary64 gradient of the composited colour with respect to points, delta, sigma, opacity
 *      and SH follows the same chain in reverse.
 *
 * Readings where the paper is silent (all of them also documented next to the settings):
 *   - q = (fx x/z + cx, fy y/z + cy); pixel (i, j) is sampled at (i + 0.5, j + 0.5).
 *   - line distances are in pixels; d = |R c + t| with c the mean of the K points (dist_mode 0)
 *     or its camera z (dist_mode 1); delta and sigma are multiplied by d^dist_power.
 *   - phi = log sum_t exp(d delta L_t) with no 1/delta normalisation; I = 1/(1 + exp(d sigma phi)).
 *   - alpha = min(alpha_max, o I); pairs with alpha < tau add nothing; compositing stops after
 *     the pair that brings the transmittance below t_min (3DGS-style constants).
 *   - the hull keeps only strictly convex vertices (collinear points and exact duplicates are
 *     dropped, lowest index kept), listed from the pivot (least v, then least u) in the order
 *     of increasing polar angle.
 *   - colour = max(0, sum_lm sh_lm Y_lm(dir) + 0.5), dir = normalise(c - camera centre).
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the discrete specification needs binary32 evaluation (FLT_EVAL_METHOD == 0)"
#endif

#define ORC_KMAX 8

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9]; /* world -> camera, row major */
    float t[3];
    float z_near;
} orc_camera;

typedef struct {
    float tau;       /* alpha below which a pair adds nothing */
    float alpha_max; /* clamp of o*I */
    float t_min;     /* stop once the transmittance falls below this, after accumulating */
    float bg[3];     /* background colour */
    int32_t dist_mode;  /* 0: d = |R c + t|, 1: d = camera z of c */
    float dist_power;   /* 0, 0.5, 1 or 2 */
    /* oracle-only knobs (no counterpart in the method):
       q_binary32 = 1 builds the hull lines from the binary32 projected points on which the hull
       was decided (the discrete specification's q), instead of a binary64 re-projection;
       perturb_ulps is the size of the conditioning probe (see render_pixels). */
    int32_t q_binary32;
    float perturb_ulps;
    /* line_rel > 0 selects the line-evaluation error model for the sensitivity bound and the
       probes: each L_t(q) may be off by line_rel (|q - a|_1 + |a - v_t|_1 + 32 + |L_t|) pixels,
       a = first hull vertex (the size of binary32 line evaluation relative to an anchor vertex);
       otherwise the vertex-motion model (every hull vertex moves by perturb_ulps ulps) is used. */
    float line_rel;
    int32_t tile_test; /* the method's exact tile test (cs_settings.tile_test) */
    /* line_f32 = 1 replaces every line value by its binary32 evaluation in record form (the lines
       kappa n_t and kappa n_t . (a - v_t) of the discrete specification, kappa = log2(e) d^p delta,
       evaluated at the pixel after re-basing them, with fused multiply-adds, to the origin of the
       pixel's 8 x 4 block), converted back to pixels with the binary64 d^p delta.  This is how a
       binary32 renderer built on that record evaluates the lines; the mode exists to check the
       line_rel error model against it (conditioning tests only). */
    int32_t line_f32;
} orc_settings;

/* flags reported per pixel by the continuous render */
#define ORC_FLAG_ALPHA_NEAR_TAU 1u  /* some evaluated alpha within ORC_ALPHA_BAND of tau */
#define ORC_FLAG_T_NEAR_TMIN 2u     /* the transmittance came within a band of t_min */
#define ORC_FLAG_CLAMP_NEAR 4u      /* some o*I within ORC_ALPHA_BAND of alpha_max */
#define ORC_ALPHA_BAND 1e-6
#define ORC_T_BAND_REL 1e-3

/* ------------------------------------------------------------------------------------------ */
/* Exact orientation of three binary32 points.                                                 */
/* Every binary32 value is m * 2^e with |m| < 2^24 and e >= -172, so each product of two is an  */
/* integer below 2^48 times 2^(e1+e2) with e1+e2 >= -344.  The sum of six such products is      */
/* formed exactly in a 640-bit fixed-point integer (positive and negative parts kept apart) and */
/* the two parts are compared.                                                                  */
/* ------------------------------------------------------------------------------------------ */
#define BIG_LIMBS 20
#define BIG_OFFSET 344

typedef struct { uint32_t w[BIG_LIMBS]; } big640;

static void big_add(big640 *b, uint64_t mag, int shift) {
    int limb = shift / 32, off = shift % 32;
    unsigned __int128 v = ((unsigned __int128)mag) << off;
    uint64_t carry = 0;
    for (int i = limb; i < BIG_LIMBS; i++) {
        uint64_t add = (uint64_t)(v & 0xffffffffu);
        v >>= 32;
        uint64_t s = (uint64_t)b->w[i] + add + carry;
        b->w[i] = (uint32_t)s;
        carry = s >> 32;
        if (v == 0 && carry == 0) break;
    }
}

static int big_cmp(const big640 *a, const big640 *b) {
    for (int i = BIG_LIMBS - 1; i >= 0; i--) {
        if (a->w[i] != b->w[i]) return a->w[i] > b->w[i] ? 1 : -1;
    }
    return 0;
}

static void f32_parts(float x, int *neg, uint64_t *mant, int *ex) {
    if (x == 0.0f) { *neg = 0; *mant = 0; *ex = 0; return; }
    int e;
    float fr = frexpf(fabsf(x), &e); /* |x| = fr * 2^e, fr in [0.5, 1) */
    *mant = (uint64_t)ldexpf(fr, 24); /* integer in [2^23, 2^24) */
    *ex = e - 24;
    *neg = x < 0.0f;
}

/* sign of sum_i s_i * a_i * b_i, computed exactly */
static int exact_sign_of_products(int n, const float *a, const float *b, const int *s) {
    big640 P, N;
    memset(&P, 0, sizeof P);
    memset(&N, 0, sizeof N);
    for (int i = 0; i < n; i++) {
        int na, nb, ea, eb;
        uint64_t ma, mb;
        f32_parts(a[i], &na, &ma, &ea);
        f32_parts(b[i], &nb, &mb, &eb);
        if (ma == 0 || mb == 0) continue;
        int neg = na ^ nb ^ (s[i] < 0);
        big_add(neg ? &N : &P, ma * mb, ea + eb + BIG_OFFSET);
    }
    return big_cmp(&P, &N);
}

/* sign of (bx-ax)(cy-ay) - (by-ay)(cx-ax) = bx cy - bx ay - ax cy - by cx + by ax + ay cx */
int orc_orient(float ax, float ay, float bx, float by, float cx, float cy) {
    const float a[6] = {bx, bx, ax, by, by, ay};
    const float b[6] = {cy, ay, cy, cx, ax, cx};
    const int s[6] = {+1, -1, -1, -1, +1, +1};
    return exact_sign_of_products(6, a, b, s);
}

/* ------------------------------------------------------------------------------------------ */
/* 2D convex hull by Graham scan (Sec. 3.2): pivot, sort by polar angle about it, then scan and */
/* remove every point that does not make a strict left turn.                                   */
/* ------------------------------------------------------------------------------------------ */
typedef struct { const float (*q)[2]; int pivot; } hull_ctx;

/* two points collinear with the pivot lie on the same ray from it (the pivot has the least v,
   ties least u), so the nearer one has the smaller v, or on a horizontal ray the smaller u */
static int nearer(const hull_ctx *h, int a, int b) {
    if (h->q[a][1] != h->q[b][1]) return h->q[a][1] < h->q[b][1];
    return h->q[a][0] < h->q[b][0];
}

static int angle_before(const hull_ctx *h, int a, int b) {
    const float (*q)[2] = h->q;
    int p = h->pivot;
    int o = orc_orient(q[p][0], q[p][1], q[a][0], q[a][1], q[b][0], q[b][1]);
    if (o != 0) return o > 0;
    return nearer(h, a, b);
}

/* returns the number T of hull vertices written to idx (T < 3 means degenerate) */
int orc_hull2d(const float *uv, int32_t k, int32_t *idx) {
    const float (*q)[2] = (const float (*)[2])uv;
    int keep[ORC_KMAX];
    if (k < 1 || k > ORC_KMAX) return 0;
    for (int i = 0; i < k; i++) {
        keep[i] = 1;
        for (int j = 0; j < i; j++)
            if (q[j][0] == q[i][0] && q[j][1] == q[i][1]) keep[i] = 0;
    }
    int p = -1;
    for (int i = 0; i < k; i++) {
        if (!keep[i]) continue;
        if (p < 0 || q[i][1] < q[p][1] || (q[i][1] == q[p][1] && q[i][0] < q[p][0])) p = i;
    }
    hull_ctx h = {q, p};
    int cand[ORC_KMAX], nc = 0;
    for (int i = 0; i < k; i++)
        if (keep[i] && i != p) cand[nc++] = i;
    for (int a = 1; a < nc; a++) { /* insertion sort by polar angle */
        int x = cand[a], b = a - 1;
        while (b >= 0 && angle_before(&h, x, cand[b])) { cand[b + 1] = cand[b]; b--; }
        cand[b + 1] = x;
    }
    int st[ORC_KMAX], ns = 0;
    st[ns++] = p;
    for (int i = 0; i < nc; i++) {
        int c = cand[i];
        while (ns >= 2 && orc_orient(q[st[ns - 2]][0], q[st[ns - 2]][1], q[st[ns - 1]][0], q[st[ns - 1]][1],
                                     q[c][0], q[c][1]) <= 0)
            ns--;
        st[ns++] = c;
    }
    for (int i = 0; i < ns; i++) idx[i] = st[i];
    return ns;
}

/* ------------------------------------------------------------------------------------------ */
/* Natural logarithm in binary32 with a fixed operation order, from the series                 */
/* ln m = 2 (s + s^3/3 + s^5/5 + ...), s = (m-1)/(m+1), after reducing x = m 2^e with m in      */
/* [sqrt(1/2), sqrt(2)).  Used only for the tile-extent radius, where both sides must agree.    */
/* ------------------------------------------------------------------------------------------ */
float orc_ln_spec(float x) {
    int e;
    float m = frexpf(x, &e);
    if (m < 0x1.6a09e6p-1f) { m = m * 2.0f; e = e - 1; }
    float num = m - 1.0f;
    float den = m + 1.0f;
    float s = num / den;
    float s2 = s * s;
    float p = 0x1.745d18p-4f;          /* 1/11 */
    p = p * s2; p = p + 0x1.c71c72p-4f; /* 1/9 */
    p = p * s2; p = p + 0x1.24924ap-3f; /* 1/7 */
    p = p * s2; p = p + 0x1.99999ap-3f; /* 1/5 */
    p = p * s2; p = p + 0x1.555556p-2f; /* 1/3 */
    p = p * s2; p = p + 1.0f;
    float two_s = 2.0f * s;
    float lnm = two_s * p;
    float eln2 = (float)e * 0x1.62e430p-1f;
    return eln2 + lnm;
}

/* ------------------------------------------------------------------------------------------ */
/* Parameter activations (Sec. 3.3): delta = exp(raw), sigma = exp(raw), o = sigmoid(raw).       */
/* The activated values decide the tile range, so both sides compute them with one fixed        */
/* binary32 definition: Cody-Waite reduction x = k ln2 + r with ln2 split into a 16-bit head    */
/* (k ln2_hi exact for |k| < 256) and a tail, |r| <= ln2/2, then the Taylor polynomial of exp r */
/* to degree 7 by Horner, scaled by 2^k.  Results below 2^-126 flush to 0, above the binary32   */
/* range they are +inf.  sigmoid(x) = 1/(1 + exp(-x)).                                         */
/* ------------------------------------------------------------------------------------------ */
float orc_exp_spec(float x) {
    if (x != x) return x;
    if (x > 88.72283935546875f) return INFINITY;
    if (x < -87.33654022216797f) return 0.0f;
    float t = x * 0x1.715476p+0f; /* log2 e */
    float k = rintf(t);
    float khi = k * 0x1.62e4p-1f;
    float klo = k * 0x1.7f7d1cp-20f;
    float r = x - khi;
    r = r - klo;
    float p = 0x1.a01a02p-13f;          /* 1/7! */
    p = p * r; p = p + 0x1.6c16c2p-10f; /* 1/6! */
    p = p * r; p = p + 0x1.111112p-7f;  /* 1/5! */
    p = p * r; p = p + 0x1.555556p-5f;  /* 1/4! */
    p = p * r; p = p + 0x1.555556p-3f;  /* 1/3! */
    p = p * r; p = p + 0.5f;
    p = p * r; p = p + 1.0f;
    p = p * r; p = p + 1.0f;
    int ki = (int)k;
    if (ki > 127) { p = p * 0x1p127f; return p * 2.0f; }
    union { uint32_t u; float f; } two_k;
    two_k.u = (uint32_t)(ki + 127) << 23;
    return p * two_k.f;
}

float orc_sigmoid_spec(float x) {
    float e = orc_exp_spec(-x);
    float den = 1.0f + e;
    return 1.0f / den;
}

/* ln_spec of n values */
void orc_ln_array(int64_t n, const float *x, float *out) {
    for (int64_t i = 0; i < n; i++) out[i] = orc_ln_spec(x[i]);
}

/* activated (delta, sigma, o) of n convexes from their raw values */
void orc_activate(int64_t n, const float *raw_delta, const float *raw_sigma, const float *raw_opacity, float *delta,
                  float *sigma, float *opacity) {
    for (int64_t i = 0; i < n; i++) {
        delta[i] = orc_exp_spec(raw_delta[i]);
        sigma[i] = orc_exp_spec(raw_sigma[i]);
        opacity[i] = orc_sigmoid_spec(raw_opacity[i]);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Exact tile test.  The rectangle bounds the mitre-offset hull {q : max_t L_t(q) <= r}, which  */
/* holds every pixel where o I >= tau; a tile of the rectangle is kept unless one hull line's  */
/* smallest value over the tile's pixel centres (a corner of [16 tx + 0.5, 16 tx + 15.5] x      */
/* [16 ty + 0.5, 16 ty + 15.5], chosen by the signs of the normal) exceeds r, so it separates  */
/* the tile from that set (a separating-axis test along the hull normals; the tile's own axes   */
/* are the rectangle).  It is evaluated on the lines as the screen record stores them,          */
/* A = kappa n_x, B = kappa n_y, C = kappa n.(anchor - v_t), kappa = d^p delta log2(e), against */
/* rk = kappa r, with a margin of 2^-20 times the magnitudes involved for binary32 rounding.   */
/* Rectangles of fewer than ORC_SAT_MIN_TILES or more than ORC_SAT_MAX_TILES tiles, and        */
/* whole-screen ones, are kept whole.                                                          */
/* ------------------------------------------------------------------------------------------ */
#define ORC_SAT_MIN_TILES 3
#define ORC_SAT_MAX_TILES 1024

static int tile_kept(const float *A, const float *B, const float *C, int T, float ax, float ay, float rk, int tx,
                     int ty) {
    float fx = (float)(16 * tx), fy = (float)(16 * ty);
    float X0 = fx + 0.5f, X1 = fx + 15.5f, Y0 = fy + 0.5f, Y1 = fy + 15.5f;
    for (int t = 0; t < T; t++) {
        float X = A[t] >= 0.0f ? X0 : X1;
        float Y = B[t] >= 0.0f ? Y0 : Y1;
        float dx = X - ax;
        float dy = Y - ay;
        float pa = A[t] * dx;
        float pb = B[t] * dy;
        float L = pa + pb;
        L = L + C[t];
        float mag = fabsf(pa) + fabsf(pb);
        mag = mag + fabsf(C[t]);
        float margin = mag * 0x1p-20f;
        float bound = rk + margin;
        if (L > bound) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Discrete specification of one convex (binary32).                                           */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int visible;
    int reason; /* 0 visible, else the first failed check (see below) */
    int full;   /* 1 if the tile range is the whole screen (degenerate mitre) */
    int T;
    int idx[ORC_KMAX];
    float uv[ORC_KMAX][2];
    uint32_t depth_bits;
    int tx0, ty0, tx1, ty1;
    int count; /* tiles kept by the exact tile test (the whole rectangle when not tested) */
    int tested;
    float lA[ORC_KMAX], lB[ORC_KMAX], lC[ORC_KMAX]; /* hull lines in record form (see below) */
    float ax, ay, rk;
} orc_disc;

enum {
    R_OK = 0, R_NONFINITE = 1, R_NONPOSITIVE = 2, R_NEAR = 3, R_RANGE = 4, R_DIST = 5,
    R_OPACITY = 6, R_HULL = 7, R_EDGE = 8, R_OFFSCREEN = 9, R_POWER = 10, R_NO_TILE = 11
};

#define ORC_COORD_LIMIT 1048576.0f /* 2^20 px */

static void xform_f32(const orc_camera *c, const float p[3], float o[3]) {
    for (int r = 0; r < 3; r++) {
        float a = c->R[3 * r + 0] * p[0];
        float b = c->R[3 * r + 1] * p[1];
        float s = a + b;
        float d = c->R[3 * r + 2] * p[2];
        s = s + d;
        o[r] = s + c->t[r];
    }
}

static int tiles_x(const orc_camera *c) { return (c->width + 15) / 16; }
static int tiles_y(const orc_camera *c) { return (c->height + 15) / 16; }

static void discrete_convex(const float *P, int K, float delta, float sigma, float opacity,
                            const orc_camera *cam, const orc_settings *st, orc_disc *out) {
    memset(out, 0, sizeof *out);
    out->reason = R_OK;
    /* 1. finite parameters */
    int finite = isfinite(delta) && isfinite(sigma) && isfinite(opacity);
    for (int i = 0; i < 3 * K; i++) finite = finite && isfinite(P[i]);
    if (!finite) { out->reason = R_NONFINITE; return; }
    if (!(delta > 0.0f) || !(sigma > 0.0f)) { out->reason = R_NONPOSITIVE; return; }
    /* 2. camera space, near plane, projection q = (fx x/z + cx, fy y/z + cy)  (Eq. 4) */
    for (int k = 0; k < K; k++) {
        float xc[3];
        xform_f32(cam, P + 3 * k, xc);
        if (!(xc[2] >= cam->z_near)) { out->reason = R_NEAR; return; }
        float xn = xc[0] / xc[2];
        float yn = xc[1] / xc[2];
        float u = cam->fx * xn;
        u = u + cam->cx;
        float v = cam->fy * yn;
        v = v + cam->cy;
        if (!(fabsf(u) <= ORC_COORD_LIMIT) || !(fabsf(v) <= ORC_COORD_LIMIT)) { out->reason = R_RANGE; return; }
        out->uv[k][0] = u;
        out->uv[k][1] = v;
    }
    /* 3. centre, camera distance (sort key) and the perspective scale d^p */
    float c[3];
    for (int a = 0; a < 3; a++) {
        float s = P[a];
        for (int k = 1; k < K; k++) s = s + P[3 * k + a];
        c[a] = s / (float)K;
    }
    float cc[3];
    xform_f32(cam, c, cc);
    float sq = cc[0] * cc[0];
    float sy = cc[1] * cc[1];
    sq = sq + sy;
    float sz = cc[2] * cc[2];
    sq = sq + sz;
    float depth = sqrtf(sq);
    float ds = st->dist_mode == 1 ? cc[2] : depth;
    if (!(ds > 0.0f) || !isfinite(ds) || !(depth > 0.0f) || !isfinite(depth)) { out->reason = R_DIST; return; }
    float g;
    if (st->dist_power == 1.0f) g = ds;
    else if (st->dist_power == 0.0f) g = 1.0f;
    else if (st->dist_power == 0.5f) g = sqrtf(ds);
    else if (st->dist_power == 2.0f) g = ds * ds;
    else { out->reason = R_POWER; return; }
    float dp = g * delta;
    float sp = g * sigma;
    memcpy(&out->depth_bits, &depth, 4);
    /* 4. opacity threshold: o*I >= tau needs o/tau - 1 > 0 (with tau = 0 every pair counts) */
    float x = 0.0f;
    int full = 0;
    if (st->tau > 0.0f) {
        float ot = opacity / st->tau;
        x = ot - 1.0f;
        if (!(x > 0.0f)) { out->reason = R_OPACITY; return; }
        if (!isfinite(x)) full = 1;
    } else {
        if (!(opacity > 0.0f)) { out->reason = R_OPACITY; return; }
        full = 1;
    }
    /* 5. hull */
    int T = orc_hull2d(&out->uv[0][0], K, out->idx);
    if (T < 3) { out->reason = R_HULL; return; }
    out->T = T;
    /* 6. outward edge normals of the hull polygon: n = (ey, -ex)/|e| */
    float nx[ORC_KMAX], ny[ORC_KMAX];
    for (int i = 0; i < T; i++) {
        const float *v = out->uv[out->idx[i]];
        const float *w = out->uv[out->idx[(i + 1) % T]];
        float ex = w[0] - v[0];
        float ey = w[1] - v[1];
        float l2 = ex * ex;
        float l2y = ey * ey;
        l2 = l2 + l2y;
        float len = sqrtf(l2);
        if (!(len > 0.0f) || !isfinite(len)) { out->reason = R_EDGE; return; }
        nx[i] = ey / len;
        ny[i] = -ex / len;
    }
    /* 7. radius r with {o I >= tau} inside {max_t L_t <= r}: from phi >= d delta max_t L_t,
          r = ln(o/tau - 1) / (d sigma * d delta); padded, then the mitre offset of the hull. */
    float r = 0.0f;
    if (!full) {
        float lnx = orc_ln_spec(x);
        float prod = sp * dp;
        r = lnx / prod;
        if (!isfinite(r)) full = 1;
    }
    if (r < 0.0f) r = 0.0f;
    float rp = r * 1.0009765625f;
    rp = rp + 0.00390625f;
    float xmin = 0, xmax = 0, ymin = 0, ymax = 0;
    for (int i = 0; i < T && !full; i++) {
        int j = (i + T - 1) % T; /* edge j ends at vertex i */
        float dot = nx[j] * nx[i];
        float doty = ny[j] * ny[i];
        dot = dot + doty;
        float den = 1.0f + dot;
        if (!(den > 0x1p-20f)) { full = 1; break; }
        float f = rp / den;
        float sx = nx[j] + nx[i];
        float syy = ny[j] + ny[i];
        float ox = f * sx;
        ox = out->uv[out->idx[i]][0] + ox;
        float oy = f * syy;
        oy = out->uv[out->idx[i]][1] + oy;
        ox = fminf(fmaxf(ox, -ORC_COORD_LIMIT), ORC_COORD_LIMIT);
        oy = fminf(fmaxf(oy, -ORC_COORD_LIMIT), ORC_COORD_LIMIT);
        if (i == 0) { xmin = xmax = ox; ymin = ymax = oy; }
        else {
            xmin = fminf(xmin, ox); xmax = fmaxf(xmax, ox);
            ymin = fminf(ymin, oy); ymax = fmaxf(ymax, oy);
        }
    }
    int ntx = tiles_x(cam), nty = tiles_y(cam);
    int tx0, tx1, ty0, ty1;
    if (full) {
        tx0 = 0; ty0 = 0; tx1 = ntx - 1; ty1 = nty - 1;
    } else {
        tx0 = (int)floorf(xmin * 0.0625f);
        tx1 = (int)floorf(xmax * 0.0625f);
        ty0 = (int)floorf(ymin * 0.0625f);
        ty1 = (int)floorf(ymax * 0.0625f);
        if (tx0 < 0) tx0 = 0;
        if (ty0 < 0) ty0 = 0;
        if (tx1 > ntx - 1) tx1 = ntx - 1;
        if (ty1 > nty - 1) ty1 = nty - 1;
    }
    if (tx0 > tx1 || ty0 > ty1 || ntx <= 0 || nty <= 0) { out->reason = R_OFFSCREEN; return; }
    out->full = full;
    out->tx0 = tx0; out->ty0 = ty0; out->tx1 = tx1; out->ty1 = ty1;
    /* 8. the record's lines: kappa = d^p delta log2 e; A, B, C relative to the anchor vertex */
    float kappa = dp * 0x1.715476p+0f;
    const float *a0 = out->uv[out->idx[0]];
    out->ax = a0[0];
    out->ay = a0[1];
    for (int t = 0; t < T; t++) {
        const float *v = out->uv[out->idx[t]];
        out->lA[t] = kappa * nx[t];
        out->lB[t] = kappa * ny[t];
        float du = a0[0] - v[0];
        float dv = a0[1] - v[1];
        float cu = nx[t] * du;
        float cv = ny[t] * dv;
        float cs = cu + cv;
        out->lC[t] = kappa * cs;
    }
    out->rk = rp * kappa;
    /* 9. tiles kept by the exact test */
    int64_t area = (int64_t)(tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    out->tested = st->tile_test && !full && area >= ORC_SAT_MIN_TILES && area <= ORC_SAT_MAX_TILES;
    if (out->tested) {
        int cnt = 0;
        for (int ty = ty0; ty <= ty1; ty++)
            for (int tx = tx0; tx <= tx1; tx++)
                cnt += tile_kept(out->lA, out->lB, out->lC, T, out->ax, out->ay, out->rk, tx, ty);
        out->count = cnt;
    } else {
        out->count = (int)area;
    }
    if (out->count == 0) { out->reason = R_NO_TILE; return; }
    out->visible = 1;
}

int orc_discrete(const float *points, int64_t n, int32_t k, const float *delta, const float *sigma,
                 const float *opacity, const orc_camera *cam, const orc_settings *st,
                 int32_t *visible, int32_t *reason, int32_t *hull_t, int32_t *hull_idx, int32_t *rect,
                 int32_t *full, uint32_t *depth_bits, float *uv, int32_t *count) {
    if (k < 3 || k > ORC_KMAX || n < 0) return -1;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        orc_disc d;
        discrete_convex(points + 3 * k * i, k, delta[i], sigma[i], opacity[i], cam, st, &d);
        if (visible) visible[i] = d.visible;
        if (reason) reason[i] = d.reason;
        if (hull_t) hull_t[i] = d.visible ? d.T : 0;
        if (hull_idx) for (int j = 0; j < ORC_KMAX; j++) hull_idx[ORC_KMAX * i + j] = (d.visible && j < d.T) ? d.idx[j] : -1;
        if (rect) {
            rect[4 * i + 0] = d.tx0; rect[4 * i + 1] = d.ty0;
            rect[4 * i + 2] = d.tx1; rect[4 * i + 3] = d.ty1;
        }
        if (full) full[i] = d.full;
        if (depth_bits) depth_bits[i] = d.depth_bits;
        if (uv) for (int j = 0; j < 2 * k; j++) uv[2 * k * i + j] = d.uv[j / 2][j % 2];
        if (count) count[i] = d.visible ? d.count : 0;
    }
    return 0;
}

/* The kept tiles (ty * tiles_x + tx, row-major within the rectangle) of every drawn convex,
   written at tiles[offsets[i] ...]; offsets come from the counts of orc_discrete. */
int orc_tiles(const float *points, int64_t n, int32_t k, const float *delta, const float *sigma,
              const float *opacity, const orc_camera *cam, const orc_settings *st, const int64_t *offsets,
              int32_t *tiles) {
    if (k < 3 || k > ORC_KMAX || n < 0) return -1;
    const int ntx = tiles_x(cam);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        orc_disc d;
        discrete_convex(points + 3 * k * i, k, delta[i], sigma[i], opacity[i], cam, st, &d);
        if (!d.visible) continue;
        int64_t o = offsets[i];
        for (int ty = d.ty0; ty <= d.ty1; ty++)
            for (int tx = d.tx0; tx <= d.tx1; tx++)
                if (!d.tested || tile_kept(d.lA, d.lB, d.lC, d.T, d.ax, d.ay, d.rk, tx, ty))
                    tiles[o++] = ty * ntx + tx;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 and their gradients (as polynomials on R^3).         */
/* ------------------------------------------------------------------------------------------ */
static void sh_basis(int deg, double x, double y, double z, double Y[16], double dY[16][3]) {
    const double pi = 3.14159265358979323846;
    const double C0 = 0.5 / sqrt(pi);
    const double C1 = sqrt(3.0 / (4.0 * pi));
    const double C2a = 0.5 * sqrt(15.0 / pi), C2b = 0.25 * sqrt(5.0 / pi), C2c = 0.25 * sqrt(15.0 / pi);
    const double C3a = 0.25 * sqrt(35.0 / (2.0 * pi)), C3b = 0.5 * sqrt(105.0 / pi);
    const double C3c = 0.25 * sqrt(21.0 / (2.0 * pi)), C3d = 0.25 * sqrt(7.0 / pi);
    const double C3e = 0.25 * sqrt(105.0 / pi);
    memset(Y, 0, 16 * sizeof(double));
    memset(dY, 0, 16 * 3 * sizeof(double));
    Y[0] = C0;
    if (deg < 1) return;
    Y[1] = -C1 * y; dY[1][1] = -C1;
    Y[2] = C1 * z;  dY[2][2] = C1;
    Y[3] = -C1 * x; dY[3][0] = -C1;
    if (deg < 2) return;
    Y[4] = C2a * x * y;  dY[4][0] = C2a * y; dY[4][1] = C2a * x;
    Y[5] = -C2a * y * z; dY[5][1] = -C2a * z; dY[5][2] = -C2a * y;
    Y[6] = C2b * (2 * z * z - x * x - y * y); dY[6][0] = -2 * C2b * x; dY[6][1] = -2 * C2b * y; dY[6][2] = 4 * C2b * z;
    Y[7] = -C2a * x * z; dY[7][0] = -C2a * z; dY[7][2] = -C2a * x;
    Y[8] = C2c * (x * x - y * y); dY[8][0] = 2 * C2c * x; dY[8][1] = -2 * C2c * y;
    if (deg < 3) return;
    Y[9] = -C3a * y * (3 * x * x - y * y);
    dY[9][0] = -6 * C3a * x * y; dY[9][1] = -C3a * (3 * x * x - 3 * y * y);
    Y[10] = C3b * x * y * z;
    dY[10][0] = C3b * y * z; dY[10][1] = C3b * x * z; dY[10][2] = C3b * x * y;
    Y[11] = -C3c * y * (4 * z * z - x * x - y * y);
    dY[11][0] = 2 * C3c * x * y; dY[11][1] = -C3c * (4 * z * z - x * x - 3 * y * y); dY[11][2] = -8 * C3c * y * z;
    Y[12] = C3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
    dY[12][0] = -6 * C3d * x * z; dY[12][1] = -6 * C3d * y * z; dY[12][2] = C3d * (6 * z * z - 3 * x * x - 3 * y * y);
    Y[13] = -C3c * x * (4 * z * z - x * x - y * y);
    dY[13][0] = -C3c * (4 * z * z - 3 * x * x - y * y); dY[13][1] = 2 * C3c * x * y; dY[13][2] = -8 * C3c * x * z;
    Y[14] = C3e * z * (x * x - y * y);
    dY[14][0] = 2 * C3e * x * z; dY[14][1] = -2 * C3e * y * z; dY[14][2] = C3e * (x * x - y * y);
    Y[15] = -C3a * x * (x * x - 3 * y * y);
    dY[15][0] = -C3a * (3 * x * x - 3 * y * y); dY[15][1] = 6 * C3a * x * y;
}

void orc_sh_basis(int32_t deg, double x, double y, double z, double *Y, double *dY) {
    double Yl[16], dYl[16][3];
    sh_basis(deg, x, y, z, Yl, dYl);
    memcpy(Y, Yl, sizeof Yl);
    if (dY) memcpy(dY, dYl, sizeof dYl);
}

/* ------------------------------------------------------------------------------------------ */
/* Continuous per-convex quantities (binary64, from the binary32 inputs).                      */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int T;
    int idx[ORC_KMAX];
    double n[ORC_KMAX][2], c0[ORC_KMAX]; /* L_t(q) = n_t . q + c0_t, outward unit normal, pixels */
    double v[ORC_KMAX][2], elen[ORC_KMAX]; /* start vertex and length of each hull edge */
    double eps;                            /* perturb_ulps binary32 ulps of the largest coordinate */
    double dp, sp;                       /* d^p delta, d^p sigma */
    double o;
    double rgb[3], raw[3];
    double r_pre; /* max_t L_t > r_pre guarantees alpha < tau - ORC_ALPHA_BAND */
    /* record-form binary32 lines and anchor (line_f32 mode), and ln 2 / (d^p delta) */
    float rA[ORC_KMAX], rB[ORC_KMAX], rC[ORC_KMAX], rax, ray;
    double s_to_px;
} orc_convex;

static uint64_t splitmix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

static void camera_centre(const orc_camera *cam, double cp[3]) {
    /* camera centre in world coordinates: -R^T t */
    for (int a = 0; a < 3; a++)
        cp[a] = -((double)cam->R[0 + a] * cam->t[0] + (double)cam->R[3 + a] * cam->t[1] + (double)cam->R[6 + a] * cam->t[2]);
}

static void xform_f64(const orc_camera *c, const double p[3], double o[3]) {
    for (int r = 0; r < 3; r++)
        o[r] = (double)c->R[3 * r] * p[0] + (double)c->R[3 * r + 1] * p[1] + (double)c->R[3 * r + 2] * p[2] + (double)c->t[r];
}

static double scale_of(const orc_settings *st, double ds) {
    if (st->dist_power == 0.0f) return 1.0;
    if (st->dist_power == 1.0f) return ds;
    if (st->dist_power == 2.0f) return ds * ds;
    return pow(ds, (double)st->dist_power);
}

static void continuous_convex(const float *P, int K, float delta, float sigma, float opacity, const float *sh,
                              int sh_deg, const orc_camera *cam, const orc_settings *st, const orc_disc *dsc,
                              uint64_t perturb_seed, int64_t id, orc_convex *cv) {
    double q[ORC_KMAX][2];
    for (int k = 0; k < K; k++) {
        if (st->q_binary32) {
            q[k][0] = dsc->uv[k][0];
            q[k][1] = dsc->uv[k][1];
        } else {
            double p[3] = {P[3 * k], P[3 * k + 1], P[3 * k + 2]}, xc[3];
            xform_f64(cam, p, xc);
            q[k][0] = (double)cam->fx * xc[0] / xc[2] + (double)cam->cx;
            q[k][1] = (double)cam->fy * xc[1] / xc[2] + (double)cam->cy;
        }
        if (perturb_seed) { /* conditioning probe: move each coordinate by perturb_ulps binary32 ulps */
            for (int a = 0; a < 2; a++) {
                uint64_t h = splitmix64(perturb_seed ^ (uint64_t)(id * 64 + k * 2 + a) * 0x2545f4914f6cdd1dull);
                float f = fabsf((float)q[k][a]);
                double ulp = (double)nextafterf(f, INFINITY) - (double)f;
                q[k][a] += ((h & 1) ? 1.0 : -1.0) * (double)st->perturb_ulps * ulp;
            }
        }
    }
    double c[3] = {0, 0, 0};
    for (int k = 0; k < K; k++)
        for (int a = 0; a < 3; a++) c[a] += P[3 * k + a];
    for (int a = 0; a < 3; a++) c[a] /= K;
    double cc[3];
    xform_f64(cam, c, cc);
    double depth = sqrt(cc[0] * cc[0] + cc[1] * cc[1] + cc[2] * cc[2]);
    double ds = st->dist_mode == 1 ? cc[2] : depth;
    double g = scale_of(st, ds);
    cv->dp = g * delta;
    cv->sp = g * sigma;
    cv->o = opacity;
    cv->T = dsc->T;
    for (int i = 0; i < dsc->T; i++) {
        cv->idx[i] = dsc->idx[i];
        const double *v = q[dsc->idx[i]];
        const double *w = q[dsc->idx[(i + 1) % dsc->T]];
        double ex = w[0] - v[0], ey = w[1] - v[1];
        double len = sqrt(ex * ex + ey * ey);
        cv->n[i][0] = ey / len;
        cv->n[i][1] = -ex / len;
        cv->c0[i] = -(cv->n[i][0] * v[0] + cv->n[i][1] * v[1]);
        cv->v[i][0] = v[0];
        cv->v[i][1] = v[1];
        cv->elen[i] = len;
    }
    {
        float big = 0.0f;
        for (int i = 0; i < dsc->T; i++)
            for (int a = 0; a < 2; a++) big = fmaxf(big, fabsf((float)cv->v[i][a]));
        cv->eps = (double)st->perturb_ulps * ((double)nextafterf(big, INFINITY) - (double)big);
    }
    double cp[3], wv[3];
    camera_centre(cam, cp);
    for (int a = 0; a < 3; a++) wv[a] = c[a] - cp[a];
    double wl = sqrt(wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]);
    double Y[16], dY[16][3];
    sh_basis(sh_deg, wv[0] / wl, wv[1] / wl, wv[2] / wl, Y, dY);
    int nb = (sh_deg + 1) * (sh_deg + 1);
    for (int ch = 0; ch < 3; ch++) {
        double s = 0.5;
        for (int j = 0; j < nb; j++) s += (double)sh[3 * j + ch] * Y[j];
        cv->raw[ch] = s;
        cv->rgb[ch] = s > 0.0 ? s : 0.0;
    }
    for (int i = 0; i < dsc->T; i++) {
        cv->rA[i] = dsc->lA[i];
        cv->rB[i] = dsc->lB[i];
        cv->rC[i] = dsc->lC[i];
    }
    cv->rax = dsc->ax;
    cv->ray = dsc->ay;
    cv->s_to_px = 0.6931471805599453 / cv->dp;
    double tl = (double)st->tau - ORC_ALPHA_BAND;
    if (tl > 0.0 && cv->o > tl)
        cv->r_pre = log(cv->o / tl - 1.0) / (cv->sp * cv->dp) * (1.0 + 1e-9) + 1e-9;
    else
        cv->r_pre = INFINITY;
}

/* ------------------------------------------------------------------------------------------ */
/* Scene preparation: discrete decisions, continuous data and the depth order.                 */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int64_t n;
    int32_t k, sh_deg;
    uint64_t probe; /* line-model probe seed (0 = none) */
    orc_disc *dsc;
    orc_convex *cv;
    int64_t *order; /* visible convexes by (depth bits, id) */
    int64_t n_order;
} orc_prepared;

static const orc_disc *g_sort_dsc;
static int cmp_order(const void *a, const void *b) {
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    uint32_t di = g_sort_dsc[i].depth_bits, dj = g_sort_dsc[j].depth_bits;
    if (di != dj) return di < dj ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}

static int prepare(orc_prepared *pr, const float *points, int64_t n, int32_t k, const float *delta,
                   const float *sigma, const float *opacity, const float *sh, int32_t sh_deg,
                   const orc_camera *cam, const orc_settings *st, uint64_t perturb_seed) {
    if (k < 3 || k > ORC_KMAX || n < 0 || sh_deg < 0 || sh_deg > 3) return -1;
    pr->n = n; pr->k = k; pr->sh_deg = sh_deg;
    pr->probe = st->line_rel > 0.0f ? perturb_seed : 0;
    pr->dsc = (orc_disc *)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_disc));
    pr->cv = (orc_convex *)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_convex));
    pr->order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!pr->dsc || !pr->cv || !pr->order) return -2;
    int nb = (sh_deg + 1) * (sh_deg + 1);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; i++) {
        discrete_convex(points + 3 * k * i, k, delta[i], sigma[i], opacity[i], cam, st, &pr->dsc[i]);
        if (pr->dsc[i].visible)
            continuous_convex(points + 3 * k * i, k, delta[i], sigma[i], opacity[i], sh + 3 * nb * i, sh_deg,
                              cam, st, &pr->dsc[i], st->line_rel > 0.0f ? 0 : perturb_seed, i, &pr->cv[i]);
    }
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (pr->dsc[i].visible) pr->order[m++] = i;
    pr->n_order = m;
    g_sort_dsc = pr->dsc;
    qsort(pr->order, (size_t)m, sizeof(int64_t), cmp_order);
    return 0;
}

static void release(orc_prepared *pr) {
    free(pr->dsc);
    free(pr->cv);
    free(pr->order);
}

/* Error model of one line value at pixel (x, y), in pixels (see line_rel / perturb_ulps). */
static double line_error(const orc_convex *cv, const orc_settings *st, double x, double y, int t, double Lt) {
    if (st->line_rel > 0.0f) {
        const double ax = cv->v[0][0], ay = cv->v[0][1];
        return (double)st->line_rel *
               (fabs(x - ax) + fabs(y - ay) + fabs(ax - cv->v[t][0]) + fabs(ay - cv->v[t][1]) + 32.0 + fabs(Lt));
    }
    /* moving the endpoints of edge t by eps moves L_t(q) by at most 2 eps (2 + |q - v_t| / |e_t|) */
    const double r = hypot(x - cv->v[t][0], y - cv->v[t][1]);
    return 2.0 * cv->eps * (2.0 + r / cv->elen[t]);
}

/* Bound on how far alpha of this pair can move under the error model: phi moves by
   d delta sum_t w_t dL_t (w = softmax weights of d delta L_t) plus the error of the
   transcendental evaluation, and alpha = o I by o I (1 - I) d sigma times the phi change. */
static double alpha_sensitivity(const orc_convex *cv, const orc_settings *st, double x, double y, const double *L,
                                double I) {
    double Lmax = -INFINITY, S = 0.0, dL = 0.0;
    for (int t = 0; t < cv->T; t++) Lmax = fmax(Lmax, L[t]);
    for (int t = 0; t < cv->T; t++) {
        double w = exp(cv->dp * (L[t] - Lmax));
        dL += w * line_error(cv, st, x, y, t, L[t]);
        S += w;
    }
    const double dphi = cv->dp * (dL / S) + 1e-6;
    return cv->o * I * (1.0 - I) * cv->sp * dphi + 1e-7;
}

/* line_f32 mode: line t at the pixel whose centre is (x, y), evaluated in binary32 from the
   record form: re-based to the pixel's 8 x 4 block origin (ox, oy) as
   C' = A (ox - a.x) + B (oy - a.y) + C, then s = A lx + B ly + C' at the pixel's offset (lx, ly)
   from that origin, each a fused multiply-add; returned in pixels (s ln 2 / (d^p delta)). */
static double line_record_f32(const orc_convex *cv, int t, double x, double y) {
    const int px = (int)floor(x), py = (int)floor(y);
    const int bx = px - px % 8, by = py - py % 4;
    const float offx = (float)bx - cv->rax, offy = (float)by - cv->ray;
    const float cp = fmaf(cv->rA[t], offx, fmaf(cv->rB[t], offy, cv->rC[t]));
    const float lx = (float)(px - bx) + 0.5f, ly = (float)(py - by) + 0.5f;
    const float s = fmaf(cv->rA[t], lx, fmaf(cv->rB[t], ly, cp));
    return (double)s * cv->s_to_px;
}

/* evaluate the smooth indicator of convex cv at pixel position (x, y); returns 0 when the pair
   is provably below tau - band (no exponentials needed), else fills phi, I and the L_t. */
static int indicator(const orc_convex *cv, const orc_settings *st, uint64_t probe, int64_t id, double x, double y,
                     double L[ORC_KMAX], double *phi, double *I) {
    double Lmax = -INFINITY;
    for (int t = 0; t < cv->T; t++) {
        L[t] = st->line_f32 ? line_record_f32(cv, t, x, y) : cv->n[t][0] * x + cv->n[t][1] * y + cv->c0[t];
        if (probe && st->line_rel > 0.0f) { /* conditioning probe of the line-evaluation model */
            uint64_t h = splitmix64(probe ^ (uint64_t)(id * 16 + t) * 0x9e3779b97f4a7c15ull);
            L[t] += ((h & 1) ? 1.0 : -1.0) * line_error(cv, st, x, y, t, L[t]);
        }
        if (L[t] > Lmax) Lmax = L[t];
    }
    if (Lmax > cv->r_pre) return 0;
    /* Eq. S1: phi = log sum_t exp(d delta L_t), evaluated around its largest term */
    double m = cv->dp * Lmax, S = 0.0;
    for (int t = 0; t < cv->T; t++) S += exp(cv->dp * L[t] - m);
    *phi = m + log(S);
    /* Eq. S2: I = Sigmoid(-d sigma phi) */
    *I = 1.0 / (1.0 + exp(cv->sp * (*phi)));
    return 1;
}

typedef struct {
    int64_t id;
    double alpha, Tb, I, phi, oI;
    double L[ORC_KMAX];
} orc_hit;

/* Eq. 5, front to back over the depth order, for one pixel.  When hits != NULL the contributing
   pairs are recorded (for the backward pass). */
static void composite(const orc_prepared *pr, const orc_settings *st, double x, double y, double rgb[3],
                      double *Tout, int64_t *last, int32_t *ncontrib, uint32_t *flags, double *sens,
                      orc_hit *hits) {
    double C[3] = {0, 0, 0}, T = 1.0, dT = 0.0, sum_Tda = 0.0;
    double cmax = fmax(fmax(fabs((double)st->bg[0]), fabs((double)st->bg[1])), fabs((double)st->bg[2]));
    int64_t lst = -1;
    int32_t nc = 0;
    uint32_t fl = 0;
    for (int64_t j = 0; j < pr->n_order; j++) {
        int64_t id = pr->order[j];
        const orc_convex *cv = &pr->cv[id];
        double L[ORC_KMAX], phi, I;
        if (!indicator(cv, st, pr->probe, id, x, y, L, &phi, &I)) continue;
        double oI = cv->o * I;
        double a = oI < (double)st->alpha_max ? oI : (double)st->alpha_max;
        /* decision bands: a fixed 1e-6 plus twice the vertex-motion sensitivity of alpha */
        double da = alpha_sensitivity(cv, st, x, y, L, I);
        double band = ORC_ALPHA_BAND + 2.0 * da;
        if (st->tau > 0.0f && fabs(a - (double)st->tau) < band) fl |= ORC_FLAG_ALPHA_NEAR_TAU;
        if (fabs(oI - (double)st->alpha_max) < band) fl |= ORC_FLAG_CLAMP_NEAR;
        if (a < (double)st->tau) continue;
        const double da_eff = a < (double)st->alpha_max ? da : 0.0;
        dT += da_eff / (1.0 - a);
        sum_Tda += T * da_eff;
        for (int ch = 0; ch < 3; ch++) cmax = fmax(cmax, cv->rgb[ch]);
        if (hits) {
            orc_hit *h = &hits[nc];
            h->id = id; h->alpha = a; h->Tb = T; h->I = I; h->phi = phi; h->oI = oI;
            memcpy(h->L, L, sizeof L);
        }
        for (int ch = 0; ch < 3; ch++) C[ch] += T * a * cv->rgb[ch];
        T *= (1.0 - a);
        lst = id;
        nc++;
        if (fabs(T - (double)st->t_min) < ORC_T_BAND_REL * (double)st->t_min + 2.0 * T * dT)
            fl |= ORC_FLAG_T_NEAR_TMIN;
        if (T < (double)st->t_min) break;
    }
    for (int ch = 0; ch < 3; ch++) rgb[ch] = C[ch] + T * (double)st->bg[ch];
    /* first-order bound on the change of any channel when the vertices move by eps:
       |dC/dalpha_n| = |T_n c_n - S_n / (1 - alpha_n)| <= 2 T_n cmax, since S_n <= T_{n+1} cmax */
    if (sens) *sens = 2.0 * cmax * sum_Tda;
    *Tout = T;
    *last = lst;
    *ncontrib = nc;
    *flags = fl;
}

int orc_render_pixels(const float *points, int64_t n, int32_t k, const float *delta, const float *sigma,
                      const float *opacity, const float *sh, int32_t sh_deg, const orc_camera *cam,
                      const orc_settings *st, const int32_t *pix, int64_t npix, uint64_t perturb_seed,
                      double *rgb, double *t_final, int64_t *last_id, int32_t *n_contrib, uint32_t *flags,
                      double *sens) {
    orc_prepared pr;
    int rc = prepare(&pr, points, n, k, delta, sigma, opacity, sh, sh_deg, cam, st, perturb_seed);
    if (rc) { release(&pr); return rc; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < npix; i++) {
        double c[3], T, sv;
        int64_t lst;
        int32_t nc;
        uint32_t fl;
        composite(&pr, st, pix[2 * i] + 0.5, pix[2 * i + 1] + 0.5, c, &T, &lst, &nc, &fl, &sv, NULL);
        if (sens) sens[i] = sv;
        for (int ch = 0; ch < 3; ch++) rgb[3 * i + ch] = c[ch];
        if (t_final) t_final[i] = T;
        if (last_id) last_id[i] = lst;
        if (n_contrib) n_contrib[i] = nc;
        if (flags) flags[i] = fl;
    }
    release(&pr);
    return 0;
}

/* Per convex, the pixel bounding box of {alpha >= tau} over the whole image (no compositing):
   used to check that the tile ranges are conservative. bbox = (x0, y0, x1, y1), or -1s if empty. */
int orc_alpha_support(const float *points, int64_t n, int32_t k, const float *delta, const float *sigma,
                      const float *opacity, const float *sh, int32_t sh_deg, const orc_camera *cam,
                      const orc_settings *st, int32_t *bbox) {
    orc_prepared pr;
    int rc = prepare(&pr, points, n, k, delta, sigma, opacity, sh, sh_deg, cam, st, 0);
    if (rc) { release(&pr); return rc; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; i++) {
        int x0 = -1, y0 = -1, x1 = -1, y1 = -1;
        if (pr.dsc[i].visible) {
            for (int y = 0; y < cam->height; y++)
                for (int x = 0; x < cam->width; x++) {
                    double L[ORC_KMAX], phi, I;
                    if (!indicator(&pr.cv[i], st, 0, i, x + 0.5, y + 0.5, L, &phi, &I)) continue;
                    double a = pr.cv[i].o * I;
                    if (a > (double)st->alpha_max) a = st->alpha_max;
                    if (a < (double)st->tau) continue;
                    if (x0 < 0 || x < x0) x0 = x;
                    if (x1 < 0 || x > x1) x1 = x;
                    if (y0 < 0 || y < y0) y0 = y;
                    if (y1 < 0 || y > y1) y1 = y;
                }
        }
        bbox[4 * i] = x0; bbox[4 * i + 1] = y0; bbox[4 * i + 2] = x1; bbox[4 * i + 3] = y1;
    }
    release(&pr);
    return 0;
}

/* per convex and tile, 1 if some pixel of the tile has binary64 alpha >= tau (mask [n][tiles]) */
int orc_alpha_tile_mask(const float *points, int64_t n, int32_t k, const float *delta, const float *sigma,
                        const float *opacity, const float *sh, int32_t sh_deg, const orc_camera *cam,
                        const orc_settings *st, uint8_t *mask) {
    orc_prepared pr;
    int rc = prepare(&pr, points, n, k, delta, sigma, opacity, sh, sh_deg, cam, st, 0);
    if (rc) { release(&pr); return rc; }
    const int ntx = tiles_x(cam), nt = ntx * tiles_y(cam);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; i++) {
        uint8_t *m = mask + (size_t)i * nt;
        memset(m, 0, (size_t)nt);
        if (!pr.dsc[i].visible) continue;
        for (int y = 0; y < cam->height; y++)
            for (int x = 0; x < cam->width; x++) {
                double L[ORC_KMAX], phi, I;
                if (!indicator(&pr.cv[i], st, 0, i, x + 0.5, y + 0.5, L, &phi, &I)) continue;
                double a = pr.cv[i].o * I;
                if (a > (double)st->alpha_max) a = st->alpha_max;
                if (a < (double)st->tau) continue;
                m[(y / 16) * ntx + x / 16] = 1;
            }
    }
    release(&pr);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Backward: analytic binary64 gradient of sum_pixels dL/dC . C with respect to the parameters. */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    double dn[ORC_KMAX][2], dc0[ORC_KMAX];
    double ddp, dsp, dop, drgb[3];
    int touched;
} orc_cgrad;

/* reverse of Eq. 5 and of the indicator for one pixel */
static void pixel_backward(const orc_prepared *pr, const orc_settings *st, double x, double y, const double G[3],
                           orc_hit *hits, orc_cgrad *cg) {
    double c[3], Tf;
    int64_t lst;
    int32_t nc;
    uint32_t fl;
    composite(pr, st, x, y, c, &Tf, &lst, &nc, &fl, NULL, hits);
    /* S accumulates, from the back, the colour seen behind the current pair: sum of later
       T_m alpha_m c_m plus T_final * bg. */
    double S[3];
    for (int ch = 0; ch < 3; ch++) S[ch] = Tf * (double)st->bg[ch];
    for (int h = nc - 1; h >= 0; h--) {
        const orc_hit *ht = &hits[h];
        const orc_convex *cv = &pr->cv[ht->id];
        orc_cgrad *g = &cg[ht->id];
        double a = ht->alpha, Tn = ht->Tb;
        /* dC/dalpha_n = T_n c_n - S / (1 - alpha_n) */
        double dalpha = 0.0;
        for (int ch = 0; ch < 3; ch++) {
            dalpha += G[ch] * (Tn * cv->rgb[ch] - S[ch] / (1.0 - a));
            g->drgb[ch] += G[ch] * Tn * a;
            S[ch] += Tn * a * cv->rgb[ch];
        }
        g->touched = 1;
        if (!(ht->oI < (double)st->alpha_max)) continue; /* clamp active: alpha is constant */
        g->dop += dalpha * ht->I;
        double dI = dalpha * cv->o;
        /* I = 1/(1+exp(sp phi)):  dI/d(sp phi) = -I (1 - I) */
        double dz = -dI * ht->I * (1.0 - ht->I);
        g->dsp += dz * ht->phi;
        double dphi = dz * cv->sp;
        /* phi = log sum exp(dp L_t): dphi/dL_t = dp w_t, dphi/d dp = sum w_t L_t */
        double Lmax = -INFINITY;
        for (int t = 0; t < cv->T; t++) if (ht->L[t] > Lmax) Lmax = ht->L[t];
        double w[ORC_KMAX], S0 = 0.0;
        for (int t = 0; t < cv->T; t++) { w[t] = exp(cv->dp * (ht->L[t] - Lmax)); S0 += w[t]; }
        for (int t = 0; t < cv->T; t++) {
            double wt = w[t] / S0;
            g->ddp += dphi * wt * ht->L[t];
            double dL = dphi * wt * cv->dp;
            g->dn[t][0] += dL * x;
            g->dn[t][1] += dL * y;
            g->dc0[t] += dL;
        }
    }
}

/* chain the per-convex gradient back to points, delta, sigma, opacity and SH */
static void convex_chain(const float *P, int K, float delta, float sigma, const float *sh, int sh_deg,
                         const orc_camera *cam, const orc_settings *st, const orc_disc *dsc, const orc_convex *cv,
                         const orc_cgrad *g, double *dP, double *ddelta, double *dsigma, double *dopa, double *dsh) {
    double xc[ORC_KMAX][3], q[ORC_KMAX][2], dq[ORC_KMAX][2];
    for (int k = 0; k < K; k++) {
        double p[3] = {P[3 * k], P[3 * k + 1], P[3 * k + 2]};
        xform_f64(cam, p, xc[k]);
        if (st->q_binary32) {
            q[k][0] = dsc->uv[k][0];
            q[k][1] = dsc->uv[k][1];
        } else {
            q[k][0] = (double)cam->fx * xc[k][0] / xc[k][2] + (double)cam->cx;
            q[k][1] = (double)cam->fy * xc[k][1] / xc[k][2] + (double)cam->cy;
        }
        dq[k][0] = dq[k][1] = 0.0;
    }
    /* lines: n = (ey, -ex)/|e|, c0 = -n.v, e = w - v */
    for (int i = 0; i < cv->T; i++) {
        int iv = cv->idx[i], iw = cv->idx[(i + 1) % cv->T];
        double vx = q[iv][0], vy = q[iv][1];
        double ex = q[iw][0] - vx, ey = q[iw][1] - vy;
        double len = sqrt(ex * ex + ey * ey);
        double nx = ey / len, ny = -ex / len;
        double dnx = g->dn[i][0] - g->dc0[i] * vx;
        double dny = g->dn[i][1] - g->dc0[i] * vy;
        dq[iv][0] += -g->dc0[i] * nx;
        dq[iv][1] += -g->dc0[i] * ny;
        double nd = nx * dnx + ny * dny;
        double dux = (dnx - nx * nd) / len, duy = (dny - ny * nd) / len;
        double dex = -duy, dey = dux; /* u = (ey, -ex) */
        dq[iw][0] += dex; dq[iw][1] += dey;
        dq[iv][0] -= dex; dq[iv][1] -= dey;
    }
    /* centre, distance, scale */
    double c[3] = {0, 0, 0};
    for (int k = 0; k < K; k++)
        for (int a = 0; a < 3; a++) c[a] += P[3 * k + a];
    for (int a = 0; a < 3; a++) c[a] /= K;
    double cc[3];
    xform_f64(cam, c, cc);
    double depth = sqrt(cc[0] * cc[0] + cc[1] * cc[1] + cc[2] * cc[2]);
    double ds = st->dist_mode == 1 ? cc[2] : depth;
    double gsc = scale_of(st, ds);
    *ddelta += g->ddp * gsc;
    *dsigma += g->dsp * gsc;
    *dopa += g->dop;
    double dg = g->ddp * delta + g->dsp * sigma;
    double pw = st->dist_power;
    double dds = pw == 0.0 ? 0.0 : dg * pw * pow(ds, pw - 1.0);
    double dcc[3] = {0, 0, 0};
    if (st->dist_mode == 1) dcc[2] = dds;
    else for (int a = 0; a < 3; a++) dcc[a] = dds * cc[a] / depth;
    double dc[3];
    for (int a = 0; a < 3; a++)
        dc[a] = (double)cam->R[a] * dcc[0] + (double)cam->R[3 + a] * dcc[1] + (double)cam->R[6 + a] * dcc[2];
    /* colour */
    double cp[3], wv[3];
    camera_centre(cam, cp);
    for (int a = 0; a < 3; a++) wv[a] = c[a] - cp[a];
    double wl = sqrt(wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2]);
    double dir[3] = {wv[0] / wl, wv[1] / wl, wv[2] / wl};
    double Y[16], dY[16][3];
    sh_basis(sh_deg, dir[0], dir[1], dir[2], Y, dY);
    int nb = (sh_deg + 1) * (sh_deg + 1);
    double ddir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ch++) {
        if (!(cv->raw[ch] > 0.0)) continue;
        double dr = g->drgb[ch];
        for (int j = 0; j < nb; j++) {
            dsh[3 * j + ch] += Y[j] * dr;
            for (int a = 0; a < 3; a++) ddir[a] += (double)sh[3 * j + ch] * dY[j][a] * dr;
        }
    }
    double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
    for (int a = 0; a < 3; a++) dc[a] += (ddir[a] - dir[a] * dd) / wl;
    /* points: through the centre (1/K each) and through the projection of hull vertices */
    for (int k = 0; k < K; k++) {
        double z = xc[k][2];
        double dx = dq[k][0] * cam->fx / z;
        double dy = dq[k][1] * cam->fy / z;
        double dz = -(dq[k][0] * cam->fx * xc[k][0] + dq[k][1] * cam->fy * xc[k][1]) / (z * z);
        for (int a = 0; a < 3; a++) {
            double dpa = (double)cam->R[a] * dx + (double)cam->R[3 + a] * dy + (double)cam->R[6 + a] * dz;
            dP[3 * k + a] += dpa + dc[a] / K;
        }
    }
}

int orc_backward_pixels(const float *points, int64_t n, int32_t k, const float *delta, const float *sigma,
                        const float *opacity, const float *sh, int32_t sh_deg, const orc_camera *cam,
                        const orc_settings *st, const int32_t *pix, int64_t npix, const double *dL_dC,
                        uint64_t perturb_seed, double *dpoints, double *ddelta, double *dsigma, double *dopacity,
                        double *dsh) {
    orc_prepared pr;
    int rc = prepare(&pr, points, n, k, delta, sigma, opacity, sh, sh_deg, cam, st, perturb_seed);
    if (rc) { release(&pr); return rc; }
    orc_cgrad *cg = (orc_cgrad *)calloc((size_t)(n > 0 ? n : 1), sizeof(orc_cgrad));
    orc_hit *hits = (orc_hit *)malloc(sizeof(orc_hit) * (size_t)(pr.n_order > 0 ? pr.n_order : 1));
    if (!cg || !hits) { free(cg); free(hits); release(&pr); return -2; }
    for (int64_t i = 0; i < npix; i++)
        pixel_backward(&pr, st, pix[2 * i] + 0.5, pix[2 * i + 1] + 0.5, dL_dC + 3 * i, hits, cg);
    int nb = (sh_deg + 1) * (sh_deg + 1);
    for (int64_t i = 0; i < n; i++) {
        if (!pr.dsc[i].visible || !cg[i].touched) continue;
        convex_chain(points + 3 * k * i, k, delta[i], sigma[i], sh + 3 * nb * i, sh_deg, cam, st, &pr.dsc[i], &pr.cv[i],
                     &cg[i],
                     dpoints + 3 * k * i, ddelta + i, dsigma + i, dopacity + i, dsh + 3 * nb * i);
    }
    free(cg);
    free(hits);
    release(&pr);
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
