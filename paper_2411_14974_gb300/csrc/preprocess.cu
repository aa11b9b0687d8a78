// Per-(view, convex) forward preprocess of the convex tile rasterizer (one thread per convex,
// points staged through shared memory with coalesced loads, SH copied asynchronously):
//   projection q_k = (fx x/z + cx, fy y/z + cy) of the K points            (Eq. 4)
//   centre c = mean p_k, camera distance d, scale d^p                       (Sec. 3.2, Eq. S1/S2)
//   exact-predicate Graham hull of the projected points                    (Sec. 3.2)
//   outward edge normals, conservative tile range, exact tile test, depth key (Sec. 3.2, 2D Eq. 1)
//   lines pre-multiplied by log2(e) d^p delta, colour from SH              (Eq. S1, Sec. 3.2)
// The decisions (visibility, hull, tile range, kept tiles, depth key) are taken in IEEE binary32
// with a fixed operation order and explicit round-to-nearest intrinsics, so they are
// reproducible bit for bit.  The block's records leave through shared memory with coalesced
// stores, and each block adds its pair count and depth-key range to the launch's totals.
#include "projection.cuh"

namespace cs {
namespace {

template <int K, int STG>
__global__ void __launch_bounds__(PRE_THREADS, 6) k_preprocess(const ViewDesc *__restrict__ views, Settings st,
                                                            PreprocessOut out) {
    // view fastest in the launch order: the blocks of every view over the same convexes run side by
    // side, so a batch of views of one scene reads the scene from HBM about once (L2 serves the rest)
    const ViewDesc &vd = views[blockIdx.x];
    const int64_t n = vd.n;
    const int64_t i0 = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * PRE_THREADS;
    if (i0 >= n) return;  // whole block
    constexpr int PS = (3 * K) | 1;  // odd stride of a convex's staged points: no bank conflicts
    __shared__ float sp[PRE_THREADS * PS];
    __shared__ __align__(16) float ssh[PRE_THREADS * SH_STAGE_WORDS];
    __shared__ float scoop[PRE_THREADS / 32][3 * KMAX + 3];
    const int cnt = (int)min((int64_t)PRE_THREADS, n - i0);
    const int shw = 3 * (vd.sh_degree + 1) * (vd.sh_degree + 1);
    // The block's SH coefficients (the bulk of its input bytes, needed last) are copied into
    // shared memory asynchronously, in their stored format, while the projection and hull run.
    const int sh_stride = stage_sh<STG>(ssh, vd.sh, i0, cnt, shw);
    {
        const int words = cnt * K * 3;
        for (int j = threadIdx.x; j < words; j += PRE_THREADS)
            sp[(j / (3 * K)) * PS + j % (3 * K)] = ld_param<STG>(vd.points, i0 * K * 3 + j);
    }
    __syncthreads();
    const int64_t i = i0 + threadIdx.x;
    const int64_t rec = vd.rec_base + i;
    const float *P = sp + threadIdx.x * PS;

    uint32_t depth_key = 0xffffffffu, count = 0, kept = 0;
    uint2 rect = make_uint2(0, 0);
    bool drawn = false, coop = false;
    float w[REC_WORDS];
    float c[3];
    float4 bbox;
    float radius = 0.f;
    int n_lines = 0;
    do {
        if (i >= n) break;
        float delta = ld_param<STG>(vd.delta, i), sigma = ld_param<STG>(vd.sigma, i);
        float opa = ld_param<STG>(vd.opacity, i);
        if (vd.activation) {
            delta = exp_act(delta);
            sigma = exp_act(sigma);
            opa = sigmoid_act(opa);
        }
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

        // ---- screen record: lines in record form, kappa = d^p delta log2(e), relative to the
        // anchor vertex; fixed rounding, since the exact tile test below runs on these values ----
        const float kappa = __fmul_rn(dp, LOG2E);
        w[R_AX] = hu[0];
        w[R_AY] = hv[0];
        w[R_SIG] = spp;
        w[R_OPA] = opa;
        w[R_HULL] = __uint_as_float(hull);
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            float A = 0.f, B = 0.f, C = 0.f;
            if (t < T) {
                A = __fmul_rn(kappa, nx[t]);
                B = __fmul_rn(kappa, ny[t]);
                C = __fmul_rn(kappa, __fadd_rn(__fmul_rn(nx[t], __fsub_rn(hu[0], hu[t])),
                                               __fmul_rn(ny[t], __fsub_rn(hv[0], hv[t]))));
            }
            w[R_LINES + 3 * t] = A;
            w[R_LINES + 3 * t + 1] = B;
            w[R_LINES + 3 * t + 2] = C;
        }
        // tiles of the rectangle kept by the exact tile test
        const float rk = __fmul_rn(rp, kappa);
        const uint32_t area = (uint32_t)(tx1 - tx0 + 1) * (uint32_t)(ty1 - ty0 + 1);
        count = area;
        kept = area <= 32u ? (area == 32u ? 0xffffffffu : (1u << area) - 1u) : 0u;
        if (st.tile_test && !full && area >= (uint32_t)SAT_MIN_TILES && area <= (uint32_t)SAT_MAX_TILES) {
            if (area <= (uint32_t)SAT_SERIAL_TILES) {
                count = 0;
                kept = 0;
                uint32_t q = 0;
                for (int ty = ty0; ty <= ty1; ++ty)
                    for (int tx = tx0; tx <= tx1; ++tx, ++q)
                        if (tile_kept(w + R_LINES, T, hu[0], hv[0], rk, tx, ty)) {
                            ++count;
                            kept |= 1u << q;
                        }
                if (count == 0) break;
            } else {
                coop = true;  // counted by the whole warp below
            }
        }
        n_lines = T;
        radius = rk;
        bbox = make_float4(xmin, ymin, xmax, ymax);
        depth_key = __float_as_uint(depth);
        rect = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
        drawn = true;
    } while (false);
    // ranges of more than SAT_SERIAL_TILES tiles: the warp tests one convex's tiles 32 at a time
    {
        const int lane = threadIdx.x & 31;
        float *slot = scoop[threadIdx.x >> 5];
        uint32_t pending = __ballot_sync(0xffffffffu, coop);
        while (pending) {
            const int src = __ffs(pending) - 1;
            pending &= pending - 1;
            if (lane == src) {  // the convex's lines, anchor and bound, for the whole warp
#pragma unroll
                for (int q = 0; q < 3 * KMAX; ++q)
                    if (q < 3 * n_lines) slot[q] = w[R_LINES + q];
                slot[3 * KMAX] = w[R_AX];
                slot[3 * KMAX + 1] = w[R_AY];
                slot[3 * KMAX + 2] = radius;
            }
            __syncwarp();
            const int Ts = __shfl_sync(0xffffffffu, n_lines, src);
            const uint32_t rx = __shfl_sync(0xffffffffu, rect.x, src), ry = __shfl_sync(0xffffffffu, rect.y, src);
            const uint32_t x0 = rx & 0xffffu, y0 = ry & 0xffffu;
            const uint32_t wd = (rx >> 16) - x0 + 1, ar = wd * ((ry >> 16) - y0 + 1);
            const float ax = slot[3 * KMAX], ay = slot[3 * KMAX + 1], rk = slot[3 * KMAX + 2];
            uint32_t n_kept = 0, first = 0;
            for (uint32_t base = 0; base < ar; base += 32) {  // warp-uniform bounds
                const uint32_t q = base + (uint32_t)lane;
                const bool keep = q < ar && tile_kept(slot, Ts, ax, ay, rk, (int)(x0 + q % wd), (int)(y0 + q / wd));
                const uint32_t b = __ballot_sync(0xffffffffu, keep);
                if (base == 0) first = b;
                n_kept += (uint32_t)__popc(b);
            }
            if (lane == src) {
                count = n_kept;
                drawn = n_kept != 0;
                kept = ar <= 32u ? first : 0u;
            }
            __syncwarp();
        }
    }
    cp_async_wait_all();
    __syncthreads();  // every thread of the block reaches this point
    if (drawn) {
        const float wx = c[0] - vd.campos[0], wy = c[1] - vd.campos[1], wz = c[2] - vd.campos[2];
        const float il = rsqrtf(wx * wx + wy * wy + wz * wz);
        const float dx = wx * il, dy = wy * il, dz = wz * il;
        const int nb = (vd.sh_degree + 1) * (vd.sh_degree + 1);
        float raw[3];
        sh_colour<STG>(ssh, threadIdx.x, shw, sh_stride, nb, dx, dy, dz, raw);
        w[R_RGB + 0] = fmaxf(raw[0], 0.f);
        w[R_RGB + 1] = fmaxf(raw[1], 0.f);
        w[R_RGB + 2] = fmaxf(raw[2], 0.f);
    }
    // The SH buffer, read by now, takes the block's records (8 chunks each at an odd stride of 9);
    // they are written out with coalesced stores below.
    constexpr int RC = REC_WORDS / 4, RS = RC + 1;
    static_assert(PRE_THREADS * RS * 4 <= PRE_THREADS * SH_STAGE_WORDS, "records fit the SH buffer");
    float4 *srec = reinterpret_cast<float4 *>(ssh);
    __shared__ uint8_t sdrawn[PRE_THREADS];
    __syncthreads();
    if (drawn) {
#pragma unroll
        for (int q = 0; q < RC; ++q)
            srec[threadIdx.x * RS + q] = make_float4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        out.bboxes[rec] = bbox;
        out.radii[rec] = radius;
        out.kept[rec] = kept;
    }
    sdrawn[threadIdx.x] = drawn ? 1 : 0;
    if (i < n) {
        out.depth_keys[rec] = drawn ? depth_key : 0xffffffffu;
        out.counts[rec] = drawn ? count : 0u;
        out.rects[rec] = drawn ? rect : make_uint2(0, 0);
    }
    // the launch's pair total and depth-key range: one set of atomics per block
    __shared__ uint32_t bsum[PRE_THREADS / 32], bmax[PRE_THREADS / 32], bmin_inv[PRE_THREADS / 32];
    const uint32_t wsum = __reduce_add_sync(0xffffffffu, drawn ? count : 0u);
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, drawn ? depth_key : 0u);
    const uint32_t wmin_inv = __reduce_max_sync(0xffffffffu, drawn ? ~depth_key : 0u);
    if ((threadIdx.x & 31) == 0) {
        bsum[threadIdx.x >> 5] = wsum;
        bmax[threadIdx.x >> 5] = wmax;
        bmin_inv[threadIdx.x >> 5] = wmin_inv;
    }
    __syncthreads();
    {
        float4 *dst = out.records + (vd.rec_base + i0) * RC;
        for (int q = threadIdx.x; q < cnt * RC; q += PRE_THREADS)
            if (sdrawn[q / RC]) dst[q] = srec[(q / RC) * RS + q % RC];
    }
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        uint32_t mx = 0, mi = 0;
#pragma unroll
        for (int q = 0; q < PRE_THREADS / 32; ++q) {
            s += bsum[q];
            mx = max(mx, bmax[q]);
            mi = max(mi, bmin_inv[q]);
        }
        if (s) {
            atomicAdd(&out.stats->pairs, s);
            atomicMax(&out.stats->key_max, mx);
            atomicMax(&out.stats->key_min_inv, mi);
        }
    }
}

}  // namespace

template <int K>
static void launch_pre_k(dim3 grid, cudaStream_t s, int storage, const ViewDesc *views_dev, const Settings &st,
                         const PreprocessOut &out) {
    if (storage == CS_STORE_F16) k_preprocess<K, CS_STORE_F16><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out);
    else if (storage == CS_STORE_BF16) k_preprocess<K, CS_STORE_BF16><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out);
    else k_preprocess<K, CS_STORE_F32><<<grid, PRE_THREADS, 0, s>>>(views_dev, st, out);
}

cudaError_t launch_preprocess(const ViewDesc *views_dev, const ViewDesc *views_host, int n_views, int64_t max_n, int k,
                              const Settings &st, const PreprocessOut &out, cudaStream_t s) {
    if (max_n <= 0 || n_views <= 0) return cudaSuccess;
    const dim3 grid = view_major_grid(n_views, max_n);
    const int storage = views_host[0].storage;  // one storage type per launch
    switch (k) {
        case 3: launch_pre_k<3>(grid, s, storage, views_dev, st, out); break;
        case 4: launch_pre_k<4>(grid, s, storage, views_dev, st, out); break;
        case 5: launch_pre_k<5>(grid, s, storage, views_dev, st, out); break;
        case 6: launch_pre_k<6>(grid, s, storage, views_dev, st, out); break;
        case 7: launch_pre_k<7>(grid, s, storage, views_dev, st, out); break;
        case 8: launch_pre_k<8>(grid, s, storage, views_dev, st, out); break;
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace cs
