// Adaptive refinement of Sec. 3.3 (details in supplement Sec. A): every convex whose sharpness
// statistic (mean |dL/dsigma| since the last refinement) exceeds a threshold is split into K
// scaled-down children centred at its K points, with sigma raised and opacity lowered; convexes
// that are too transparent or too large are pruned.  Decisions and child values are binary32
// expressions with a fixed operation order (the CPU side mirrors them bit for bit).
//
// Two kernels around a device-wide scan: k_refine_decide writes each convex's decision and its
// output count (0, 1 or K), the exclusive scan gives output offsets and the total, and
// k_refine_scatter writes kept convexes (with their Adam moments) and children (moments 0).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/convex_splat.h"
#include "cs_api_internal.h"
#include "cs_spec_math.cuh"

using namespace cs;

namespace {

constexpr int REF_THREADS = 128;

struct RefineArgs {
    cs_param_arrays in, m, v, out, om, ov;
    const float *stat;
    int64_t n;
    int k, shw;
    float window;  // the mean statistic is a binary32 division by the window length
    float threshold, split_scale, sigma_scale, opacity_scale, prune_opacity, prune_size;
};

__device__ __forceinline__ void centre_of(const float *P, int K, float c[3]) {
    for (int a = 0; a < 3; ++a) {
        float s = P[a];
        for (int k = 1; k < K; ++k) s = __fadd_rn(s, P[3 * k + a]);
        c[a] = __fdiv_rn(s, (float)K);
    }
}

__global__ void __launch_bounds__(REF_THREADS) k_refine_decide(const RefineArgs a, int32_t *__restrict__ decision,
                                                               uint32_t *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * REF_THREADS + threadIdx.x;
    if (i >= a.n) return;
    const float *P = a.in.points + i * a.k * 3;
    float c[3];
    centre_of(P, a.k, c);
    float size = 0.f;
    bool finite = true;
    for (int k = 0; k < a.k; ++k) {
        const float dx = __fsub_rn(P[3 * k], c[0]), dy = __fsub_rn(P[3 * k + 1], c[1]),
                    dz = __fsub_rn(P[3 * k + 2], c[2]);
        const float r = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
        finite = finite && (r == r);
        size = fmaxf(size, r);
    }
    const float o = sigmoid_act(a.in.opacity[i]);
    const float mean = __fdiv_rn(a.stat[i], a.window);
    int d;
    if (!finite || !(o >= a.prune_opacity) || !(size <= a.prune_size)) d = 2;
    else if (mean > a.threshold) d = 1;
    else d = 0;
    if (decision) decision[i] = d;
    count[i] = d == 2 ? 0u : (d == 1 ? (uint32_t)a.k : 1u);
}

__device__ __forceinline__ void copy_row(const float *src, float *dst, int64_t i, int w) {
    if (!src || !dst) return;
    for (int q = 0; q < w; ++q) dst[i * w + q] = src[i * w + q];
}

__device__ __forceinline__ void zero_row(float *dst, int64_t i, int w) {
    if (!dst) return;
    for (int q = 0; q < w; ++q) dst[i * w + q] = 0.f;
}

__global__ void __launch_bounds__(REF_THREADS) k_refine_scatter(const RefineArgs a, const uint32_t *__restrict__ count,
                                                                const uint32_t *__restrict__ offset) {
    const int64_t i = (int64_t)blockIdx.x * REF_THREADS + threadIdx.x;
    if (i >= a.n) return;
    const uint32_t cnt = count[i];
    if (cnt == 0) return;
    const int64_t o = offset[i];
    const int pw = a.k * 3;
    if (cnt == 1) {  // kept: parameters and moments move to their new slot
        const cs_param_arrays *src[3] = {&a.in, &a.m, &a.v};
        const cs_param_arrays *dst[3] = {&a.out, &a.om, &a.ov};
        for (int s = 0; s < 3; ++s) {
            const cs_param_arrays &S = *src[s];
            const cs_param_arrays &D = *dst[s];
            if (!S.points || !D.points) continue;
            for (int q = 0; q < pw; ++q) D.points[o * pw + q] = S.points[i * pw + q];
            D.delta[o] = S.delta[i];
            D.sigma[o] = S.sigma[i];
            D.opacity[o] = S.opacity[i];
            for (int q = 0; q < a.shw; ++q) D.sh[o * a.shw + q] = S.sh[i * a.shw + q];
        }
        return;
    }
    // split into K children
    const float *P = a.in.points + i * pw;
    float c[3];
    centre_of(P, a.k, c);
    const float op = sigmoid_act(a.in.opacity[i]);
    const float oc = __fmul_rn(op, a.opacity_scale);
    const float child_opacity = ln_series(__fdiv_rn(oc, __fsub_rn(1.0f, oc)));
    const float child_sigma = __fadd_rn(a.in.sigma[i], ln_series(a.sigma_scale));
    const float delta = a.in.delta[i];
    for (int j = 0; j < a.k; ++j) {
        const int64_t t = o + j;
        for (int k = 0; k < a.k; ++k)
            for (int ax = 0; ax < 3; ++ax)
                a.out.points[t * pw + 3 * k + ax] =
                    __fadd_rn(P[3 * j + ax], __fmul_rn(a.split_scale, __fsub_rn(P[3 * k + ax], c[ax])));
        a.out.delta[t] = delta;
        a.out.sigma[t] = child_sigma;
        a.out.opacity[t] = child_opacity;
        for (int q = 0; q < a.shw; ++q) a.out.sh[t * a.shw + q] = a.in.sh[i * a.shw + q];
        const cs_param_arrays *mo[2] = {&a.om, &a.ov};
        for (int s = 0; s < 2; ++s) {
            const cs_param_arrays &D = *mo[s];
            if (!D.points) continue;
            for (int q = 0; q < pw; ++q) D.points[t * pw + q] = 0.f;
            D.delta[t] = 0.f;
            D.sigma[t] = 0.f;
            D.opacity[t] = 0.f;
            for (int q = 0; q < a.shw; ++q) D.sh[t * a.shw + q] = 0.f;
        }
    }
}

bool complete(const cs_param_arrays *p) {
    return p && p->points && p->delta && p->sigma && p->opacity && p->sh;
}

}  // namespace

extern "C" cs_status cs_refine(cs_context *ctx, int64_t n, int32_t k, int32_t sh_degree, const cs_param_arrays *params,
                               const cs_param_arrays *adam_m, const cs_param_arrays *adam_v,
                               const float *sigma_grad_abs, int32_t window_steps, const cs_refine_settings *st,
                               int64_t capacity, cs_param_arrays *out_params, cs_param_arrays *out_m,
                               cs_param_arrays *out_v, int32_t *decisions, int64_t *n_out, void *stream_ptr) {
    if (!ctx || !st || !n_out) return fail(CS_ERR_ARG, "context, settings or n_out is NULL");
    *n_out = 0;
    if (n < 0 || n > ((int64_t)1 << 31) / KMAX) return fail(CS_ERR_ARG, "n = %lld out of range", (long long)n);
    if (k < 3 || k > KMAX) return fail(CS_ERR_ARG, "k = %d: 3 <= k <= 8", k);
    if (sh_degree < 0 || sh_degree > 3) return fail(CS_ERR_ARG, "sh_degree must be 0..3");
    if (window_steps < 1) return fail(CS_ERR_ARG, "window_steps must be >= 1");
    if ((adam_m == nullptr) != (adam_v == nullptr) || (adam_m == nullptr) != (out_m == nullptr) ||
        (out_m == nullptr) != (out_v == nullptr))
        return fail(CS_ERR_ARG, "Adam moments: give adam_m, adam_v, out_m and out_v, or none of them");
    if (!(st->split_scale > 0.f) || !(st->split_sigma_scale > 0.f) || !(st->split_opacity_scale > 0.f) ||
        !(st->split_opacity_scale <= 1.f))
        return fail(CS_ERR_ARG, "split scales must be positive (opacity scale <= 1)");
    if (n == 0) return CS_OK;
    if (!complete(params) || !sigma_grad_abs || !out_params || !complete(out_params) ||
        (adam_m && (!complete(adam_m) || !complete(adam_v) || !complete(out_m) || !complete(out_v))))
        return fail(CS_ERR_ARG, "a parameter or moment array is NULL");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream_ptr;
    RefineArgs a{};
    a.in = *params;
    if (adam_m) {
        a.m = *adam_m;
        a.v = *adam_v;
        a.om = *out_m;
        a.ov = *out_v;
    }
    a.out = *out_params;
    a.stat = sigma_grad_abs;
    a.n = n;
    a.k = k;
    a.shw = 3 * (sh_degree + 1) * (sh_degree + 1);
    a.window = (float)window_steps;
    a.threshold = st->split_threshold;
    a.split_scale = st->split_scale;
    a.sigma_scale = st->split_sigma_scale;
    a.opacity_scale = st->split_opacity_scale;
    a.prune_opacity = st->prune_opacity;
    a.prune_size = st->prune_size;
    uint32_t *count = nullptr, *offset = nullptr;
    unsigned long long *tmp = nullptr, *total = nullptr;
    const unsigned blocks = (unsigned)((n + REF_THREADS - 1) / REF_THREADS);
    cs_status code = CS_OK;
    unsigned long long total_h = 0;
    cudaError_t e = pool_alloc(ctx, (void **)&count, (size_t)n * 4, s);
    if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&offset, (size_t)n * 4, s);
    if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&tmp, scan_tmp_words(n) * 8 + 16, s);
    if (e == cudaSuccess) {
        total = tmp + scan_tmp_words(n);
        k_refine_decide<<<blocks, REF_THREADS, 0, s>>>(a, decisions, count);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_exclusive_scan(count, nullptr, offset, n, total, tmp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total_h, total, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        *n_out = (int64_t)total_h;
        if ((int64_t)total_h > capacity) {
            code = fail(CS_ERR_BUDGET, "refinement yields %llu convexes, capacity %lld", total_h, (long long)capacity);
        } else if (total_h > 0) {
            k_refine_scatter<<<blocks, REF_THREADS, 0, s>>>(a, count, offset);
            count_launches(1);
            e = cudaGetLastError();
        }
    }
    pool_free(count, s);
    pool_free(offset, s);
    pool_free(tmp, s);
    if (e != cudaSuccess) return fail_cuda(e, "cs_refine");
    return code;
}
