// Per-(view, convex) backward preprocess of the convex tile rasterizer: one thread per drawn
// convex applies the chain rule from the per-record gradient accumulated by the blend backward
// (lines, sigma', opacity, colour) to the hull vertices, the projected points, the 3D points
// (Eq. 4 Jacobian), delta, sigma, the camera distance (Eq. S1/S2), the opacity and the SH
// coefficients, and, for training parameters, through the exp / sigmoid activations (Sec. 3.3).
#include "projection.cuh"

namespace cs {
namespace {

// Backward: one thread per drawn convex.  The block's SH coefficients are staged in shared memory
// (coalesced asynchronous copy, conflict-free layout).  With one view, the points and SH gradients
// of the block's convexes are gathered in shared memory and added to the outputs with coalesced
// accesses (binary32 SH: each thread overwrites its own staged coefficients with their gradients
// once it has read them); with several views, convexes are shared between views and use global
// atomics.
template <int K, int DEG, bool ATOMIC, int STG>
__global__ void __launch_bounds__(PRE_THREADS, 5) k_preprocess_backward(const ViewDesc *__restrict__ views, Settings st,
                                                                     const float4 *__restrict__ records,
                                                                     const uint32_t *__restrict__ counts,
                                                                     const float4 *__restrict__ grads,
                                                                     PreprocessGrads out) {
    constexpr int NB = (DEG + 1) * (DEG + 1);
    constexpr int PW = K * 3, SW = NB * 3;           // words per convex
    // the block's point gradients are staged contiguously (as in the output, so that they leave
    // with 16-byte stores); the separate 16-bit-storage SH gradients at an odd stride (no bank
    // conflicts)
    constexpr int PS = PW, SS = SW | 1;
    constexpr int esz = STG == CS_STORE_F32 ? 4 : 2;
    constexpr bool CHUNKED = (SW * esz) % 16 == 0;   // degrees 1 and 3: 16-byte chunk layout possible
    constexpr bool IN_PLACE = !ATOMIC && STG == CS_STORE_F32;  // SH gradients overwrite the staged SH
    constexpr bool SEP_DSH = !ATOMIC && STG != CS_STORE_F32;   // 16-bit SH: a separate binary32 buffer
    __shared__ float s_dp[ATOMIC ? 1 : PRE_THREADS * PS];
    __shared__ __align__(16) float ssh[PRE_THREADS * (STG == CS_STORE_F32 ? SH_STAGE_WORDS : SH_STAGE_WORDS / 2 + 2)];
    __shared__ float s_dsh[SEP_DSH ? PRE_THREADS * SS : 1];
    // view fastest in the launch order (see k_preprocess)
    const ViewDesc &vd = views[blockIdx.x];
    const int64_t i0 = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * PRE_THREADS;
    if (i0 >= vd.n) return;
    const int cnt = (int)min((int64_t)PRE_THREADS, vd.n - i0);
    const int sh_stride = stage_sh<STG>(ssh, vd.sh, i0, cnt, SW);
    if (!ATOMIC) {  // the gradients to add to: the buffers' contents, or zero when they are written
        if (out.dpoints)
            for (int q = threadIdx.x; q < cnt * PW; q += PRE_THREADS) s_dp[q] = out.write ? 0.f : out.dpoints[i0 * PW + q];
        if (SEP_DSH && out.dsh)
            for (int q = threadIdx.x; q < cnt * SW; q += PRE_THREADS)
                s_dsh[(q / SW) * SS + q % SW] = out.write ? 0.f : out.dsh[i0 * SW + q];
    }
    // slot of SH word w of this thread's convex in the staged buffer (binary32 words)
    auto sh_slot = [&](int w) -> float & {
        float *base = ssh + (sh_stride ? threadIdx.x * sh_stride * 4 : threadIdx.x * SW);
        return base[w];
    };
    auto zero_sh_slots = [&]() {
        if (IN_PLACE) {
#pragma unroll
            for (int w = 0; w < SW; ++w) sh_slot(w) = 0.f;
        }
    };
    const int64_t i = i0 + threadIdx.x;
    const int64_t rec = vd.rec_base + i;
    // the lines this thread reads after the barrier (its gradient record, the record's colour and
    // hull, its points) and the block's SH gradients updated at the end are requested into L2 while
    // the block waits for its staged SH
    if (i < vd.n) {
        prefetch_l2(grads + rec * (GRAD_WORDS / 4));
        prefetch_l2(records + rec * (REC_WORDS / 4));
        const char *pp = reinterpret_cast<const char *>(vd.points) + (size_t)i * PW * esz;
        prefetch_l2(pp);
        prefetch_l2(pp + PW * esz - 1);
    }
    if (IN_PLACE && out.dsh && !out.write)
        for (int q = threadIdx.x * 32; q < cnt * SW; q += PRE_THREADS * 32) prefetch_l2(out.dsh + i0 * SW + q);
    const bool live = i < vd.n && counts[rec] != 0;
    if (!ATOMIC && out.write && i < vd.n && !live) {  // a convex that is not drawn: zero gradients
        if (out.ddelta) out.ddelta[i] = 0.f;
        if (out.dsigma) out.dsigma[i] = 0.f;
        if (out.dopacity) out.dopacity[i] = 0.f;
    }
    cp_async_wait_all();
    __syncthreads();  // staged SH (and, with one view, the gathered gradients) visible to the block
    if (!live && i < vd.n) zero_sh_slots();
    if (live) {
        float gw[GRAD_WORDS];
        const float4 h0 = records[rec * (REC_WORDS / 4)], h1 = records[rec * (REC_WORDS / 4) + 1];
#pragma unroll
        for (int q = 0; q < GRAD_WORDS / 4; ++q) {
            const float4 b = grads[rec * (GRAD_WORDS / 4) + q];
            gw[4 * q] = b.x; gw[4 * q + 1] = b.y; gw[4 * q + 2] = b.z; gw[4 * q + 3] = b.w;
        }
        (void)h0;
        static_assert(R_RGB == 4 && R_HULL == 7, "colour and hull in the record's second float4");
        const uint32_t hull = __float_as_uint(h1.w);
        const int T = (int)hull_pack_count(hull);
        float delta = ld_param<STG>(vd.delta, i), sigma = ld_param<STG>(vd.sigma, i);
        if (vd.activation) {
            delta = exp_act(delta);
            sigma = exp_act(sigma);
        }
        float p[K][3], xc[K][3], u[K], v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            p[k][0] = ld_param<STG>(vd.points, i * PW + 3 * k);
            p[k][1] = ld_param<STG>(vd.points, i * PW + 3 * k + 1);
            p[k][2] = ld_param<STG>(vd.points, i * PW + 3 * k + 2);
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
        float hu[K], hv[K];
#pragma unroll
        for (int t = 0; t < K; ++t)
            if (t < T) select_point<K>(u, v, hull_pack_index(hull, t), hu[t], hv[t]);
        const float ax = hu[0], ay = hv[0];
        float dkappa = 0.f;
        float dhu[K], dhv[K];
#pragma unroll
        for (int t = 0; t < K; ++t) dhu[t] = dhv[t] = 0.f;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            if (t >= T) break;
            const int t1 = (t + 1 == T) ? 0 : t + 1;
            float wx = hu[0], wy = hv[0];
#pragma unroll
            for (int q = 1; q < K; ++q)
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
            for (int q = 0; q < K; ++q)
                if (q == t1) { dhu[q] += dex; dhv[q] += dey; }
            dhu[t] -= dex;
            dhv[t] -= dey;
        }
        float du[K], dv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) du[k] = dv[k] = 0.f;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            if (t >= T) break;
            const int k = hull_pack_index(hull, t);
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (q == k) { du[q] += dhu[t]; dv[q] += dhv[t]; }
        }
        // delta, sigma, opacity, distance
        const float gsig = gw[G_SIG];
        float dd_delta = dkappa * g * LOG2E, dd_sigma = gsig * g, dd_opa = gw[G_OPA];
        if (vd.activation) {  // to the raw values: d exp = exp, d sigmoid = o (1 - o)
            const float o = sigmoid_act(ld_param<STG>(vd.opacity, i));
            dd_delta *= delta;
            dd_sigma *= sigma;
            dd_opa *= o * (1.0f - o);
        }
        if (ATOMIC) {
            if (out.ddelta && dd_delta != 0.f) atomicAdd(out.ddelta + i, dd_delta);
            if (out.dsigma && dd_sigma != 0.f) atomicAdd(out.dsigma + i, dd_sigma);
            if (out.dopacity && dd_opa != 0.f) atomicAdd(out.dopacity + i, dd_opa);
        } else if (out.write) {
            if (out.ddelta) out.ddelta[i] = dd_delta;
            if (out.dsigma) out.dsigma[i] = dd_sigma;
            if (out.dopacity) out.dopacity[i] = dd_opa;
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
            // the record holds max(raw, 0) per channel, so it is positive exactly where the clamp
            // passes the gradient
            const float gr[3] = {h1.x > 0.f ? gw[G_RGB] : 0.f, h1.y > 0.f ? gw[G_RGB + 1] : 0.f,
                                 h1.z > 0.f ? gw[G_RGB + 2] : 0.f};
            float ddx = 0.f, ddy = 0.f, ddz = 0.f;
            // dL/dc_jc = Y_j gr_c; the direction gradient sums (sum_c c_jc gr_c) dY_j/dd
            auto emit = [&](int j, int c, float d) {
                if (ATOMIC) {
                    if (out.dsh && d != 0.f) atomicAdd(out.dsh + i * SW + 3 * j + c, d);
                } else if (SEP_DSH) {
                    s_dsh[threadIdx.x * SS + 3 * j + c] += d;
                }
            };
            if (gr[0] != 0.f || gr[1] != 0.f || gr[2] != 0.f) {
                if (CHUNKED && sh_stride) {
                    constexpr int EPC = 16 / esz;  // elements per chunk
                    uint4 *s4 = reinterpret_cast<uint4 *>(ssh) + threadIdx.x * sh_stride;
                    uint4 ch = make_uint4(0u, 0u, 0u, 0u);
                    float dch[4];
#pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        float gx, gy, gz;
                        const float Yj = sh_term(j, dx, dy, dz, gx, gy, gz);
                        float sg = 0.f;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const int w = 3 * j + c;
                            if (w % EPC == 0) ch = s4[w / EPC];
                            sg += chunk_elem<STG>(ch, w % EPC) * gr[c];
                            const float d = Yj * gr[c];
                            emit(j, c, d);
                            if (IN_PLACE) {  // the chunk's four words are read before it is overwritten
                                dch[w % 4] = d;
                                if (w % 4 == 3) s4[w / 4] = make_uint4(__float_as_uint(dch[0]), __float_as_uint(dch[1]),
                                                                       __float_as_uint(dch[2]), __float_as_uint(dch[3]));
                            }
                        }
                        if (DEG > 0) {
                            ddx += sg * gx;
                            ddy += sg * gy;
                            ddz += sg * gz;
                        }
                    }
                } else {
                    const int sb = threadIdx.x * SW;
#pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        float gx, gy, gz;
                        const float Yj = sh_term(j, dx, dy, dz, gx, gy, gz);
                        float sg = 0.f;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            sg += sm_param<STG>(ssh, sb + 3 * j + c) * gr[c];
                            const float d = Yj * gr[c];
                            emit(j, c, d);
                            if (IN_PLACE) ssh[sb + 3 * j + c] = d;
                        }
                        if (DEG > 0) {
                            ddx += sg * gx;
                            ddy += sg * gy;
                            ddz += sg * gz;
                        }
                    }
                }
            } else {
                zero_sh_slots();
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
        if (out.dpoints) {
            // 16-byte stores from where the block's range starts on a 16-byte boundary
            float *dst = out.dpoints + i0 * PW;
            const int n = cnt * PW;
            const int head = min(n, (int)(((16u - ((uintptr_t)dst & 15u)) & 15u) / 4u));
            const int n4 = (n - head) / 4;
            for (int q = threadIdx.x; q < head; q += PRE_THREADS) dst[q] = s_dp[q];
            float4 *d4 = reinterpret_cast<float4 *>(dst + head);
            for (int q = threadIdx.x; q < n4; q += PRE_THREADS)
                d4[q] = make_float4(s_dp[head + 4 * q], s_dp[head + 4 * q + 1], s_dp[head + 4 * q + 2],
                                    s_dp[head + 4 * q + 3]);
            for (int q = head + 4 * n4 + threadIdx.x; q < n; q += PRE_THREADS) dst[q] = s_dp[q];
        }
        if (out.dsh) {
            float *dst = out.dsh + i0 * SW;
            if (IN_PLACE && sh_stride && ((uintptr_t)dst & 15u) == 0) {
                // the staged chunks (sh_stride 16-byte chunks per convex) leave with 16-byte stores
                constexpr int C = SW / 4;
                const uint4 *s4 = reinterpret_cast<const uint4 *>(ssh);
                float4 *d4 = reinterpret_cast<float4 *>(dst);
                for (int f = threadIdx.x; f < cnt * C; f += PRE_THREADS) {
                    const int t = f / C;
                    const uint4 v = s4[t * sh_stride + (f - t * C)];
                    float4 d = make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z),
                                           __uint_as_float(v.w));
                    if (!out.write) {
                        const float4 o = d4[f];
                        d.x += o.x; d.y += o.y; d.z += o.z; d.w += o.w;
                    }
                    d4[f] = d;
                }
            } else if (IN_PLACE) {
                for (int q = threadIdx.x; q < cnt * SW; q += PRE_THREADS) {
                    const int t = q / SW;
                    const float d = sh_stride ? ssh[t * sh_stride * 4 + (q - t * SW)] : ssh[q];
                    if (out.write) out.dsh[i0 * SW + q] = d;
                    else out.dsh[i0 * SW + q] += d;
                }
            } else {
                for (int q = threadIdx.x; q < cnt * SW; q += PRE_THREADS)
                    out.dsh[i0 * SW + q] = s_dsh[(q / SW) * SS + q % SW];
            }
        }
    }
}

}  // namespace

template <int K, int STG>
static void launch_pre_bwd_k(dim3 grid, cudaStream_t s, int deg, bool atomic, const ViewDesc *views_dev,
                             const Settings &st, const float4 *records, const uint32_t *counts, const float4 *grads,
                             const PreprocessGrads &g) {
#define CS_PRE_BWD(D, A) \
    k_preprocess_backward<K, D, A, STG><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, records, counts, grads, g)
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

template <int K>
static void launch_pre_bwd_ks(dim3 grid, cudaStream_t s, int storage, int deg, bool atomic,
                              const ViewDesc *views_dev, const Settings &st, const float4 *records,
                              const uint32_t *counts, const float4 *grads, const PreprocessGrads &g) {
    if (storage == CS_STORE_F16)
        launch_pre_bwd_k<K, CS_STORE_F16>(grid, s, deg, atomic, views_dev, st, records, counts, grads, g);
    else if (storage == CS_STORE_BF16)
        launch_pre_bwd_k<K, CS_STORE_BF16>(grid, s, deg, atomic, views_dev, st, records, counts, grads, g);
    else
        launch_pre_bwd_k<K, CS_STORE_F32>(grid, s, deg, atomic, views_dev, st, records, counts, grads, g);
}

cudaError_t launch_preprocess_backward(const ViewDesc *views_dev, int n_views, int64_t max_n, int k, int sh_degree,
                                       int storage, const Settings &st, const float4 *records, const uint32_t *counts,
                                       const float4 *grad_records, const PreprocessGrads &g, bool atomic,
                                       cudaStream_t s) {
    if (max_n <= 0 || n_views <= 0) return cudaSuccess;
    if (sh_degree < 0 || sh_degree > 3) return cudaErrorInvalidValue;
    const dim3 grid = view_major_grid(n_views, max_n);
    switch (k) {
        case 3:
            launch_pre_bwd_ks<3>(grid, s, storage, sh_degree, atomic, views_dev, st, records, counts, grad_records, g);
            break;
        case 4:
            launch_pre_bwd_ks<4>(grid, s, storage, sh_degree, atomic, views_dev, st, records, counts, grad_records, g);
            break;
        case 5:
            launch_pre_bwd_ks<5>(grid, s, storage, sh_degree, atomic, views_dev, st, records, counts, grad_records, g);
            break;
        case 6:
            launch_pre_bwd_ks<6>(grid, s, storage, sh_degree, atomic, views_dev, st, records, counts, grad_records, g);
            break;
        case 7:
            launch_pre_bwd_ks<7>(grid, s, storage, sh_degree, atomic, views_dev, st, records, counts, grad_records, g);
            break;
        case 8:
            launch_pre_bwd_ks<8>(grid, s, storage, sh_degree, atomic, views_dev, st, records, counts, grad_records, g);
            break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace cs
