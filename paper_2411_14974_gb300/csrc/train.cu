// Training step around the renderer (Sec. 3.3): the photometric loss (1 - lambda) L1 +
// lambda D-SSIM of Eq. 6 (without the mask term) with its gradient, and the Adam update.
//
// SSIM (Wang et al. 2004) uses an 11 x 11 Gaussian window (sd 1.5, separable, normalised),
// C1 = 0.01^2, C2 = 0.03^2 and zero padding outside the image, per channel plane.  With the
// local moments mu_x = G*x, E_xx = G*(x x), E_xy = G*(x y) (and likewise for y),
//   S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
// s_xx = E_xx - mu_x^2, s_xy = E_xy - mu_x mu_y.  The gradient of sum S w.r.t. x is
//   G*a + 2 x (G*b) + y (G*c),  a = dS/dmu_x, b = dS/dE_xx, c = dS/dE_xy
// (the window is symmetric, so the adjoint of the zero-padded correlation is the same filter).
// Both kernels stage a 32 x 16 output tile plus a 5-pixel halo in shared memory and filter it
// separably (rows, then columns); the forward writes a, b, c and block sums of S and |x - y|,
// the backward filters a, b, c and forms dL/dx.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/convex_splat.h"
#include "cs_api_internal.h"

using namespace cs;

namespace {

constexpr int SSIM_TW = 32, SSIM_TH = 16, SSIM_R = 5, SSIM_TAPS = 2 * SSIM_R + 1;
constexpr int SSIM_LW = SSIM_TW + 2 * SSIM_R, SSIM_LH = SSIM_TH + 2 * SSIM_R;
constexpr int SSIM_THREADS = 256;
constexpr float SSIM_C1 = 0.01f * 0.01f, SSIM_C2 = 0.03f * 0.03f;

struct Gauss {
    float w[SSIM_TAPS];
};

__device__ __forceinline__ float block_sum(float v, float *red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < SSIM_THREADS / 32; ++i) s += red[i];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(SSIM_THREADS) k_ssim_forward(const float *__restrict__ x, const float *__restrict__ y,
                                                               int H, int W, Gauss g, float *__restrict__ amap,
                                                               float *__restrict__ bmap, float *__restrict__ cmap,
                                                               double *__restrict__ sums) {
    __shared__ float sx[SSIM_LH][SSIM_LW], sy[SSIM_LH][SSIM_LW];
    __shared__ float hs[5][SSIM_LH][SSIM_TW];
    __shared__ float red[SSIM_THREADS / 32];
    const size_t plane = (size_t)blockIdx.z * H * W;
    const int ox = blockIdx.x * SSIM_TW, oy = blockIdx.y * SSIM_TH;
    for (int q = threadIdx.x; q < SSIM_LH * SSIM_LW; q += SSIM_THREADS) {
        const int r = q / SSIM_LW, c = q % SSIM_LW;
        const int gy = oy - SSIM_R + r, gx = ox - SSIM_R + c;
        float vx = 0.f, vy = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            vx = __ldg(x + plane + (size_t)gy * W + gx);
            vy = __ldg(y + plane + (size_t)gy * W + gx);
        }
        sx[r][c] = vx;
        sy[r][c] = vy;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SSIM_LH * SSIM_TW; q += SSIM_THREADS) {
        const int r = q / SSIM_TW, c = q % SSIM_TW;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f, m4 = 0.f;
#pragma unroll
        for (int k = 0; k < SSIM_TAPS; ++k) {
            const float a = sx[r][c + k], b = sy[r][c + k], w = g.w[k];
            m0 += w * a;
            m1 += w * b;
            m2 += w * a * a;
            m3 += w * b * b;
            m4 += w * a * b;
        }
        hs[0][r][c] = m0; hs[1][r][c] = m1; hs[2][r][c] = m2; hs[3][r][c] = m3; hs[4][r][c] = m4;
    }
    __syncthreads();
    const int c = threadIdx.x & 31;
    float sum_s = 0.f, sum_l1 = 0.f;
    for (int r = threadIdx.x >> 5; r < SSIM_TH; r += SSIM_THREADS / 32) {
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < SSIM_TAPS; ++k) {
            const float w = g.w[k];
#pragma unroll
            for (int j = 0; j < 5; ++j) m[j] += w * hs[j][r + k][c];
        }
        const int gy = oy + r, gx = ox + c;
        if (gy < H && gx < W) {
            const float mx = m[0], my = m[1];
            const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
            const float A1 = 2.f * mx * my + SSIM_C1, A2 = 2.f * sxy + SSIM_C2;
            const float B1 = mx * mx + my * my + SSIM_C1, B2 = sxx + syy + SSIM_C2;
            const float iD = 1.0f / (B1 * B2);
            const float S = A1 * A2 * iD;
            const float d_mx = 2.f * (my * A2 - S * mx * B2) * iD;
            const float d_sxx = -S * B1 * iD;
            const float d_sxy = 2.f * A1 * iD;
            const size_t o = plane + (size_t)gy * W + gx;
            amap[o] = d_mx - 2.f * mx * d_sxx - my * d_sxy;
            bmap[o] = d_sxx;
            cmap[o] = d_sxy;
            sum_s += S;
            sum_l1 += fabsf(sx[r + SSIM_R][c + SSIM_R] - sy[r + SSIM_R][c + SSIM_R]);
        }
    }
    const float bs = block_sum(sum_s, red);
    const float bl = block_sum(sum_l1, red);
    if (threadIdx.x == 0) {
        atomicAdd(sums, (double)bs);
        atomicAdd(sums + 1, (double)bl);
    }
}

__global__ void __launch_bounds__(SSIM_THREADS) k_ssim_backward(const float *__restrict__ x, const float *__restrict__ y,
                                                                int H, int W, Gauss g, const float *__restrict__ amap,
                                                                const float *__restrict__ bmap,
                                                                const float *__restrict__ cmap, float l1_scale,
                                                                float ssim_scale, float *__restrict__ dx) {
    __shared__ float sa[3][SSIM_LH][SSIM_LW];
    __shared__ float hs[3][SSIM_LH][SSIM_TW];
    const size_t plane = (size_t)blockIdx.z * H * W;
    const int ox = blockIdx.x * SSIM_TW, oy = blockIdx.y * SSIM_TH;
    for (int q = threadIdx.x; q < SSIM_LH * SSIM_LW; q += SSIM_THREADS) {
        const int r = q / SSIM_LW, c = q % SSIM_LW;
        const int gy = oy - SSIM_R + r, gx = ox - SSIM_R + c;
        float va = 0.f, vb = 0.f, vc = 0.f;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
            const size_t o = plane + (size_t)gy * W + gx;
            va = __ldg(amap + o);
            vb = __ldg(bmap + o);
            vc = __ldg(cmap + o);
        }
        sa[0][r][c] = va;
        sa[1][r][c] = vb;
        sa[2][r][c] = vc;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < SSIM_LH * SSIM_TW; q += SSIM_THREADS) {
        const int r = q / SSIM_TW, c = q % SSIM_TW;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
#pragma unroll
        for (int k = 0; k < SSIM_TAPS; ++k) {
            const float w = g.w[k];
            m0 += w * sa[0][r][c + k];
            m1 += w * sa[1][r][c + k];
            m2 += w * sa[2][r][c + k];
        }
        hs[0][r][c] = m0; hs[1][r][c] = m1; hs[2][r][c] = m2;
    }
    __syncthreads();
    const int c = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < SSIM_TH; r += SSIM_THREADS / 32) {
        const int gy = oy + r, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        float fa = 0.f, fb = 0.f, fc = 0.f;
#pragma unroll
        for (int k = 0; k < SSIM_TAPS; ++k) {
            const float w = g.w[k];
            fa += w * hs[0][r + k][c];
            fb += w * hs[1][r + k][c];
            fc += w * hs[2][r + k][c];
        }
        const size_t o = plane + (size_t)gy * W + gx;
        const float xv = __ldg(x + o), yv = __ldg(y + o);
        const float d = xv - yv;
        const float sgn = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
        dx[o] = l1_scale * sgn - ssim_scale * (fa + 2.f * xv * fb + yv * fc);
    }
}

__global__ void k_loss_finalize(const double *sums, double count, float lambda, float *loss_out) {
    const double l1 = sums[1] / count, s = sums[0] / count;
    *loss_out = (float)((1.0 - (double)lambda) * l1 + (double)lambda * (1.0 - s));
}

// ---- Adam ------------------------------------------------------------------------------------
constexpr int ADAM_THREADS = 256, ADAM_PER_THREAD = 4, ADAM_CHUNK = ADAM_THREADS * ADAM_PER_THREAD * 4;

struct AdamGroupDev {
    float *p, *g, *m, *v, *acc;
    int64_t n;
    float lr;
    int vec4;  // every pointer 16-byte aligned: float4 access
};

struct AdamArgs {
    AdamGroupDev grp[CS_ADAM_MAX_GROUPS];
    int64_t first_block[CS_ADAM_MAX_GROUPS + 1];
    int n_groups;
    float b1, b2, eps, bc1, bc2;  // bc = 1 / (1 - beta^t)
    int zero_grad;
};

__device__ __forceinline__ void adam_one(const AdamArgs &a, float lr, float &p, float &g, float &m, float &v) {
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * g * g;
    const float mhat = m * a.bc1, vhat = v * a.bc2;
    p = p - lr * mhat / (sqrtf(vhat) + a.eps);
}

__global__ void __launch_bounds__(ADAM_THREADS) k_adam(const AdamArgs a) {
    int gi = 0;
    while (gi + 1 < a.n_groups && (int64_t)blockIdx.x >= a.first_block[gi + 1]) ++gi;
    const AdamGroupDev &G = a.grp[gi];
    const int64_t base = ((int64_t)blockIdx.x - a.first_block[gi]) * ADAM_CHUNK;
    const int64_t end = min(G.n, base + ADAM_CHUNK);
    if (G.vec4 && end - base == ADAM_CHUNK) {
        float4 *P = (float4 *)(G.p + base), *Gr = (float4 *)(G.g + base), *M = (float4 *)(G.m + base),
               *Vv = (float4 *)(G.v + base);
        float4 *Ac = G.acc ? (float4 *)(G.acc + base) : nullptr;
#pragma unroll
        for (int u = 0; u < ADAM_PER_THREAD; ++u) {
            const int q = threadIdx.x + u * ADAM_THREADS;
            float4 p = P[q], g = Gr[q], m = M[q], v = Vv[q];
            if (Ac) {
                float4 s = Ac[q];
                s.x += fabsf(g.x); s.y += fabsf(g.y); s.z += fabsf(g.z); s.w += fabsf(g.w);
                Ac[q] = s;
            }
            adam_one(a, G.lr, p.x, g.x, m.x, v.x);
            adam_one(a, G.lr, p.y, g.y, m.y, v.y);
            adam_one(a, G.lr, p.z, g.z, m.z, v.z);
            adam_one(a, G.lr, p.w, g.w, m.w, v.w);
            P[q] = p; M[q] = m; Vv[q] = v;
            if (a.zero_grad) Gr[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        for (int64_t i = base + threadIdx.x; i < end; i += ADAM_THREADS) {
            float p = G.p[i], g = G.g[i], m = G.m[i], v = G.v[i];
            if (G.acc) G.acc[i] += fabsf(g);
            adam_one(a, G.lr, p, g, m, v);
            G.p[i] = p; G.m[i] = m; G.v[i] = v;
            if (a.zero_grad) G.g[i] = 0.f;
        }
    }
}

Gauss gauss_window() {
    Gauss g;
    double w[SSIM_TAPS], s = 0.0;
    for (int k = 0; k < SSIM_TAPS; ++k) {
        const double d = k - SSIM_R;
        w[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        s += w[k];
    }
    for (int k = 0; k < SSIM_TAPS; ++k) g.w[k] = (float)(w[k] / s);
    return g;
}

}  // namespace

extern "C" cs_status cs_loss_l1_dssim(cs_context *ctx, const float *image, const float *target, int32_t n_views,
                                      int32_t height, int32_t width, float lambda, float *loss_out, float *dL_dimage,
                                      void *stream_ptr) {
    if (!ctx) return fail(CS_ERR_ARG, "context is NULL");
    if (n_views < 0 || height < 0 || width < 0) return fail(CS_ERR_ARG, "negative image size");
    if (!(lambda >= 0.f && lambda <= 1.f)) return fail(CS_ERR_ARG, "lambda must be in [0, 1]");
    const int64_t planes = (int64_t)n_views * 3, M = planes * height * width;
    if (M == 0) return CS_OK;
    if (!image || !target) return fail(CS_ERR_ARG, "image or target is NULL");
    if (planes > 65535) return fail(CS_ERR_ARG, "at most 21845 views per call");
    if (!loss_out && !dL_dimage) return CS_OK;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream_ptr;
    StageTimer tm(ctx, CS_STAGE_LOSS, s);
    float *maps = nullptr;
    double *sums = nullptr;
    cudaError_t e = pool_alloc(ctx, (void **)&maps, (size_t)M * 3 * sizeof(float), s);
    if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&sums, 2 * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
    const Gauss g = gauss_window();
    const dim3 grid((unsigned)((width + SSIM_TW - 1) / SSIM_TW), (unsigned)((height + SSIM_TH - 1) / SSIM_TH),
                    (unsigned)planes);
    if (e == cudaSuccess) {
        k_ssim_forward<<<grid, SSIM_THREADS, 0, s>>>(image, target, height, width, g, maps, maps + M, maps + 2 * M,
                                                     sums);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && loss_out) {
        k_loss_finalize<<<1, 1, 0, s>>>(sums, (double)M, lambda, loss_out);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && dL_dimage) {
        k_ssim_backward<<<grid, SSIM_THREADS, 0, s>>>(image, target, height, width, g, maps, maps + M, maps + 2 * M,
                                                      (float)((1.0 - lambda) / (double)M), (float)(lambda / (double)M),
                                                      dL_dimage);
        count_launches(1);
        e = cudaGetLastError();
    }
    pool_free(maps, s);
    pool_free(sums, s);
    return e == cudaSuccess ? CS_OK : fail_cuda(e, "cs_loss_l1_dssim");
}

extern "C" cs_status cs_adam_step(cs_context *ctx, const cs_adam_group *groups, int32_t n_groups,
                                  const cs_adam_settings *st, int64_t step, void *stream_ptr) {
    if (!ctx) return fail(CS_ERR_ARG, "context is NULL");
    if (!st) return fail(CS_ERR_ARG, "settings is NULL");
    if (n_groups < 0 || n_groups > CS_ADAM_MAX_GROUPS) return fail(CS_ERR_ARG, "0..%d groups", CS_ADAM_MAX_GROUPS);
    if (n_groups > 0 && !groups) return fail(CS_ERR_ARG, "groups is NULL");
    if (step < 1) return fail(CS_ERR_ARG, "step counts from 1");
    if (!(st->beta1 >= 0.f && st->beta1 < 1.f) || !(st->beta2 >= 0.f && st->beta2 < 1.f) || !(st->eps >= 0.f))
        return fail(CS_ERR_ARG, "0 <= beta < 1 and eps >= 0 required");
    AdamArgs a{};
    a.b1 = st->beta1;
    a.b2 = st->beta2;
    a.eps = st->eps;
    a.bc1 = (float)(1.0 / (1.0 - std::pow((double)st->beta1, (double)step)));
    a.bc2 = (float)(1.0 / (1.0 - std::pow((double)st->beta2, (double)step)));
    a.zero_grad = st->zero_grad != 0;
    int64_t blocks = 0;
    int ng = 0;
    for (int i = 0; i < n_groups; ++i) {
        const cs_adam_group &G = groups[i];
        if (G.n < 0) return fail(CS_ERR_ARG, "group %d: negative size", i);
        if (G.n == 0) continue;
        if (!G.param || !G.grad || !G.m || !G.v) return fail(CS_ERR_ARG, "group %d has a NULL buffer", i);
        AdamGroupDev &D = a.grp[ng];
        D.p = G.param; D.g = G.grad; D.m = G.m; D.v = G.v; D.acc = G.grad_abs_sum;
        D.n = G.n;
        D.lr = G.lr;
        uintptr_t any = (uintptr_t)G.param | (uintptr_t)G.grad | (uintptr_t)G.m | (uintptr_t)G.v |
                        (uintptr_t)G.grad_abs_sum;
        D.vec4 = (any & 15) == 0;
        a.first_block[ng] = blocks;
        blocks += (G.n + ADAM_CHUNK - 1) / ADAM_CHUNK;
        ++ng;
    }
    a.first_block[ng] = blocks;
    a.n_groups = ng;
    if (blocks == 0) return CS_OK;
    if (blocks > 0x7fffffff) return fail(CS_ERR_ARG, "too many elements");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream_ptr;
    StageTimer tm(ctx, CS_STAGE_OPTIMIZER, s);
    k_adam<<<(unsigned)blocks, ADAM_THREADS, 0, s>>>(a);
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CS_OK : fail_cuda(e, "cs_adam_step");
}
