// C-ABI entry points of the convex tile rasterizer: context, forward, backward, state access.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "cs_api_internal.h"
#include "cs_common.cuh"

using namespace cs;

// ---------------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------------
static thread_local char g_err[512] = "";

cs_status cs::fail(cs_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

cs_status cs::fail_cuda(cudaError_t e, const char *what) {
    cudaGetLastError();  // clear a sticky launch error so the next call starts clean
    return fail(CS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *cs_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------------------------
// instrumentation: launch counter and per-stage events
// ---------------------------------------------------------------------------------------------
static std::atomic<uint64_t> g_launches{0};
void cs::count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
extern "C" uint64_t cs_kernel_launch_count(void) { return g_launches.load(); }

static cudaEvent_t take_event(cs_context *ctx) {
    cudaEvent_t e = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->prof_mu);
        if (!ctx->free_events.empty()) {
            e = ctx->free_events.back();
            ctx->free_events.pop_back();
        }
    }
    if (!e && cudaEventCreate(&e) != cudaSuccess) e = nullptr;
    return e;
}

cs::StageTimer::StageTimer(cs_context *ctx, int stage, cudaStream_t s) : ctx_(ctx), stage_(stage), s_(s) {
    if (ctx_ && ctx_->profiling) {
        a_ = take_event(ctx_);
        if (a_) cudaEventRecord(a_, s_);
    }
}

cs::StageTimer::~StageTimer() {
    if (!a_) return;
    cudaEvent_t b = take_event(ctx_);
    if (!b) return;
    cudaEventRecord(b, s_);
    std::lock_guard<std::mutex> lk(ctx_->prof_mu);
    ctx_->prof.push_back({stage_, a_, b});
}

extern "C" cs_status cs_profile_enable(cs_context *ctx, int32_t on) {
    if (!ctx) return fail(CS_ERR_ARG, "context is NULL");
    ctx->profiling = on != 0;
    return CS_OK;
}

extern "C" cs_status cs_profile_read(cs_context *ctx, double *ms, int64_t *launches) {
    if (!ctx) return fail(CS_ERR_ARG, "context is NULL");
    std::vector<cs_context::StageRec> recs;
    {
        std::lock_guard<std::mutex> lk(ctx->prof_mu);
        recs.swap(ctx->prof);
    }
    for (int i = 0; i < CS_STAGE_COUNT; ++i) {
        if (ms) ms[i] = 0.0;
        if (launches) launches[i] = 0;
    }
    cs_status st = CS_OK;
    for (auto &r : recs) {
        cudaError_t e = cudaEventSynchronize(r.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess && st == CS_OK) st = fail_cuda(e, "profile events");
        if (r.stage >= 0 && r.stage < CS_STAGE_COUNT) {
            if (ms) ms[r.stage] += t;
            if (launches) launches[r.stage] += 1;
        }
        std::lock_guard<std::mutex> lk(ctx->prof_mu);
        ctx->free_events.push_back(r.a);
        ctx->free_events.push_back(r.b);
    }
    return st;
}

extern "C" void cs_default_settings(cs_settings *s) {
    if (!s) return;
    s->tau = 1.0f / 255.0f;
    s->alpha_max = 0.99f;
    s->t_min = 1e-4f;
    s->bg[0] = s->bg[1] = s->bg[2] = 0.f;
    s->dist_mode = 0;
    s->dist_power = 1.0f;
    s->tile_test = 0;
    s->tile_split = 0;
}

// ---------------------------------------------------------------------------------------------
// context and stream-ordered allocations
// ---------------------------------------------------------------------------------------------
extern "C" cs_status cs_context_create(int32_t device, cs_context **out) {
    if (!out) return fail(CS_ERR_ARG, "cs_context_create: out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) return fail(CS_ERR_ARG, "device %d out of range (%d devices)", device, count);
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDeviceProperties");
    if (prop.major * 10 + prop.minor != 103)
        return fail(CS_ERR_CUDA, "device %d is sm_%d%d; this library is built for sm_103a only", device, prop.major,
                    prop.minor);
    int prev = 0;
    cudaGetDevice(&prev);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaSetDevice");
    cs_context *c = new (std::nothrow) cs_context();
    if (!c) return fail(CS_ERR_NOMEM, "out of host memory");
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&c->pool, &props);
    if (e != cudaSuccess) {
        delete c;
        cudaSetDevice(prev);
        return fail_cuda(e, "cudaMemPoolCreate");
    }
    uint64_t keep = UINT64_MAX;  // keep freed memory in the pool: later calls reuse it without the driver
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    // the readback slots are written by a kernel (no copy engine), through their device address
    e = cudaHostAlloc(&c->host_total, sizeof(unsigned long long) * 8, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&c->host_total_dev, c->host_total, 0);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->totals_ready, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (c->host_total) cudaFreeHost(c->host_total);
        cudaMemPoolDestroy(c->pool);
        delete c;
        cudaSetDevice(prev);
        return fail_cuda(e, "context set-up");
    }
    cudaSetDevice(prev);
    *out = c;
    return CS_OK;
}

extern "C" void cs_context_destroy(cs_context *ctx) {
    if (!ctx) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    // first the worker of the pipelined host-buffer steps: it enqueues what is queued (using the
    // context's pool, events and profiling records), then ends
    if (ctx->host_worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(ctx->job_mu);
            ctx->worker_stop = true;
        }
        ctx->job_cv.notify_all();
        ctx->host_worker.join();
    }
    cudaDeviceSynchronize();
    for (auto &r : ctx->prof) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->free_events) cudaEventDestroy(e);
    for (auto &sl : ctx->host_slots) {
        if (sl.buf) cudaFree(sl.buf);
        if (sl.uploaded) cudaEventDestroy(sl.uploaded);
        if (sl.computed) cudaEventDestroy(sl.computed);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (ctx->upload_stream) cudaStreamDestroy(ctx->upload_stream);
    if (ctx->compute_stream) cudaStreamDestroy(ctx->compute_stream);
    if (ctx->download_stream) cudaStreamDestroy(ctx->download_stream);
    if (ctx->host_total) cudaFreeHost(ctx->host_total);
    if (ctx->totals_ready) cudaEventDestroy(ctx->totals_ready);
    cudaMemPoolTrimTo(ctx->pool, 0);
    cudaMemPoolDestroy(ctx->pool);
    cudaSetDevice(prev);
    delete ctx;
}

// Allocation sizes above 1 MiB are rounded up to one of eight sizes per power of two (at most
// 12.5% more): buffers whose sizes change a little from call to call (the pair lists of different
// views) then reuse the pool's blocks instead of making it map more memory, which takes the host
// about a millisecond per call.
static size_t size_class(size_t bytes) {
    if (bytes <= ((size_t)1 << 20)) return (bytes + 255) & ~(size_t)255;
    const int lg = 63 - __builtin_clzll((unsigned long long)bytes);
    const size_t q = (size_t)1 << (lg - 3);
    return (bytes + q - 1) & ~(q - 1);
}

cudaError_t cs::pool_alloc(cs_context *ctx, void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    bytes = size_class(bytes);
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, s);
#if CS_CHECKED
    // checked builds hand out every buffer filled with 0xff bytes (NaN as float): a read of a
    // buffer before it is written then shows in the results
    if (e == cudaSuccess) e = fill_words(*p, 0xffffffffu, bytes, s);
#endif
    return e;
}

cs_status cs::take_device_status(cudaStream_t s, const char *what) {
#if CS_CHECKED
    unsigned bits = 0;
    cudaError_t e = take_status_blend(&bits, s);
    if (e == cudaSuccess) e = take_status_sort(&bits, s);
    if (e != cudaSuccess) return fail_cuda(e, what);
    if (bits)
        return fail(CS_ERR_DEVICE, "%s: device status 0x%x (1 tile range, 2 record index, 4 hull count, 8 pair slot, "
                    "16 tile index, 32 sort slot outside its buffer; the accesses were skipped)", what, bits);
#else
    (void)s;
    (void)what;
#endif
    return CS_OK;
}

void cs::pool_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------------------------------------
// validation helpers
// ---------------------------------------------------------------------------------------------
cs_status cs::check_settings(const cs_settings *st) {
    if (!st) return fail(CS_ERR_ARG, "settings is NULL");
    if (!(st->tau >= 0.f && st->tau < 1.f)) return fail(CS_ERR_ARG, "tau must be in [0, 1)");
    if (!(st->alpha_max > 0.f && st->alpha_max <= 1.f)) return fail(CS_ERR_ARG, "alpha_max must be in (0, 1]");
    if (!(st->t_min >= 0.f && st->t_min < 1.f)) return fail(CS_ERR_ARG, "t_min must be in [0, 1)");
    if (st->dist_mode != 0 && st->dist_mode != 1) return fail(CS_ERR_ARG, "dist_mode must be 0 or 1");
    if (st->tile_test != 0 && st->tile_test != 1) return fail(CS_ERR_ARG, "tile_test must be 0 or 1");
    if (st->tile_split != 0 && (st->tile_split < 256 || st->tile_split > (1 << 24)))
        return fail(CS_ERR_ARG, "tile_split must be 0 or in 256..2^24 pairs");
    const float p = st->dist_power;
    if (!(p == 0.f || p == 0.5f || p == 1.f || p == 2.f)) return fail(CS_ERR_ARG, "dist_power must be 0, 0.5, 1 or 2");
    for (int i = 0; i < 3; ++i)
        if (!isfinite(st->bg[i])) return fail(CS_ERR_ARG, "bg must be finite");
    return CS_OK;
}

cs_status cs::check_camera(const cs_camera *c) {
    if (c->width <= 0 || c->height <= 0 || c->width > 32768 || c->height > 32768)
        return fail(CS_ERR_ARG, "camera size %dx%d out of range (1..32768)", c->width, c->height);
    const float v[] = {c->fx, c->fy, c->cx, c->cy, c->z_near};
    for (float x : v)
        if (!isfinite(x)) return fail(CS_ERR_ARG, "camera intrinsics must be finite");
    for (int i = 0; i < 9; ++i)
        if (!isfinite(c->R[i])) return fail(CS_ERR_ARG, "camera R must be finite");
    for (int i = 0; i < 3; ++i)
        if (!isfinite(c->t[i])) return fail(CS_ERR_ARG, "camera t must be finite");
    if (!(c->z_near > 0.f)) return fail(CS_ERR_ARG, "z_near must be > 0");
    return CS_OK;
}

cs_status cs::check_scene(const cs_scene *s) {
    if (!s) return fail(CS_ERR_ARG, "scene is NULL");
    if (s->n < 0 || s->n > (int64_t)1 << 31) return fail(CS_ERR_ARG, "scene size %lld out of range", (long long)s->n);
    if (s->k < 3 || s->k > KMAX) return fail(CS_ERR_ARG, "k = %d: 3 <= k <= 8 points per convex", s->k);
    if (s->sh_degree < 0 || s->sh_degree > 3) return fail(CS_ERR_ARG, "sh_degree must be 0..3");
    if (s->activation != CS_ACT_NONE && s->activation != CS_ACT_EXP_SIGMOID)
        return fail(CS_ERR_ARG, "activation must be CS_ACT_NONE or CS_ACT_EXP_SIGMOID");
    if (s->storage != CS_STORE_F32 && s->storage != CS_STORE_F16 && s->storage != CS_STORE_BF16)
        return fail(CS_ERR_ARG, "storage must be CS_STORE_F32, CS_STORE_F16 or CS_STORE_BF16");
    if (s->n > 0 && (!s->points || !s->delta || !s->sigma || !s->opacity || !s->sh))
        return fail(CS_ERR_ARG, "scene has a NULL buffer");
    return CS_OK;
}

void cs::fill_view(ViewDesc &vd, const cs_camera &c) {
    memset(&vd, 0, sizeof vd);
    memcpy(vd.R, c.R, sizeof vd.R);
    memcpy(vd.t, c.t, sizeof vd.t);
    vd.fx = c.fx; vd.fy = c.fy; vd.cx = c.cx; vd.cy = c.cy; vd.z_near = c.z_near;
    for (int a = 0; a < 3; ++a)
        vd.campos[a] = (float)(-((double)c.R[a] * c.t[0] + (double)c.R[3 + a] * c.t[1] + (double)c.R[6 + a] * c.t[2]));
    vd.width = c.width;
    vd.height = c.height;
    vd.tiles_x = (c.width + TILE - 1) / TILE;
    vd.tiles_y = (c.height + TILE - 1) / TILE;
}

Settings cs::to_settings(const cs_settings &s) {
    Settings o;
    o.tau = s.tau; o.alpha_max = s.alpha_max; o.t_min = s.t_min;
    o.bg[0] = s.bg[0]; o.bg[1] = s.bg[1]; o.bg[2] = s.bg[2];
    o.dist_mode = s.dist_mode; o.dist_power = s.dist_power;
    o.tile_test = s.tile_test;
    o.tile_split = s.tile_split;
    return o;
}

// ---------------------------------------------------------------------------------------------
// forward pipeline over a batch of views
// ---------------------------------------------------------------------------------------------
#define CS_TRY(expr, what)                               \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) {                         \
            st_code = fail_cuda(_e, what);               \
            goto cleanup;                                \
        }                                                \
    } while (0)

void cs::state_free(cs_fwd_state *s) {
    if (!s) return;
    cudaStream_t st = s->stream;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->ctx->device);
    pool_free(s->views_dev, st);
    pool_free(s->records, st);
    pool_free(s->depth_keys, st);
    pool_free(s->rects, st);
    pool_free(s->counts, st);
    pool_free(s->bboxes, st);
    pool_free(s->pair_keys, st);
    pool_free(s->pair_vals, st);
    pool_free(s->ranges, st);
    pool_free(s->n_last, st);
    pool_free(s->t_final_own, st);
    pool_free(s->tile_order, st);
    pool_free(s->split_items, st);
    pool_free(s->split_heavy, st);
    pool_free(s->split_slot, st);
    pool_free(s->chunk_state, st);
    cudaSetDevice(prev);
    delete s;
}

// the tile-split fields of the blend arguments, from a forward state (none when not split)
static void set_split_args(BlendArgs &a, const cs_fwd_state *s) {
    a.tile_order = s->tile_order;
    if (!s->split_items) return;
    a.split = (uint32_t)s->st.tile_split;
    a.split_items = s->split_items;
    a.n_items = s->n_items;
    a.split_heavy = s->split_heavy;
    a.n_heavy = s->n_heavy;
    a.split_slot = s->split_slot;
    a.chunk_state = s->chunk_state;
}

static int bits_for(uint64_t n) {
    int b = 0;
    while (b < 32 && ((uint64_t)1 << b) < n) ++b;
    return b;
}

cs_status cs::run_forward(cs_context *ctx, cs_fwd_state *s, cudaStream_t stream) {
    cs_status st_code = CS_OK;
    const int V = (int)s->views.size();
    int64_t R = 0, max_n = 0;
    uint32_t tiles = 0;
    for (int v = 0; v < V; ++v) {
        ViewDesc &vd = s->views[v];
        vd.rec_base = R;
        vd.tile_base = tiles;
        R += vd.n;
        max_n = vd.n > max_n ? vd.n : max_n;
        tiles += (uint32_t)(vd.tiles_x * vd.tiles_y);
    }
    s->n_records = R;
    s->n_tiles = tiles;
    s->stream = stream;
    size_t pix_total = 0;
    for (int v = 0; v < V; ++v) pix_total += (size_t)s->views[v].width * s->views[v].height;

    uint32_t *sort_keys_a = nullptr, *sort_keys_b = nullptr, *sort_vals_a = nullptr, *sort_vals_b = nullptr;
    uint32_t *offsets = nullptr, *radix_tmp = nullptr, *pk_b = nullptr, *pv_b = nullptr;
    unsigned long long *scan_tmp = nullptr, *total = nullptr;
    float *radii = nullptr;
    uint64_t P = 0;
    int depth_bits = 0;
    bool in_b = false;
    // one persistent blend launch over all views, with a completion flag per view (serving loop)
    const bool persist = s->view_flags && s->st.tile_split == 0 && V <= MAX_ORDER_VIEWS &&
                         s->view_done.size() == (size_t)V;
    uint32_t max_view_tiles = 1;
    for (int v = 0; v < V; ++v) {
        const uint32_t t = (uint32_t)(s->views[v].tiles_x * s->views[v].tiles_y);
        max_view_tiles = t > max_view_tiles ? t : max_view_tiles;
    }
    const int local_bits = bits_for(max_view_tiles);
    const int view_bits = bits_for((uint64_t)V);
    if (local_bits + view_bits > 32) return fail(CS_ERR_ARG, "too many views and tiles for a 32-bit pair key");
    s->local_bits = local_bits;
    // block masks ride in the pair keys' free high bits when there are enough of them
    s->mask_shift = local_bits + view_bits + BLOCK_MASK_BITS <= 32 ? local_bits + view_bits : 0;

    CS_TRY(pool_alloc(ctx, (void **)&s->views_dev, sizeof(ViewDesc) * V, stream), "alloc views");
    CS_TRY(pool_alloc(ctx, (void **)&s->records, (size_t)R * REC_WORDS * 4, stream), "alloc records");
    CS_TRY(pool_alloc(ctx, (void **)&s->depth_keys, (size_t)R * 4, stream), "alloc depth keys");
    CS_TRY(pool_alloc(ctx, (void **)&s->rects, (size_t)R * 8, stream), "alloc rects");
    CS_TRY(pool_alloc(ctx, (void **)&s->counts, (size_t)R * 4, stream), "alloc counts");
    CS_TRY(pool_alloc(ctx, (void **)&s->bboxes, (size_t)R * 16, stream), "alloc boxes");
    CS_TRY(pool_alloc(ctx, (void **)&radii, (size_t)R * 8, stream), "alloc radii");  // radii, kept masks
    CS_TRY(pool_alloc(ctx, (void **)&s->ranges, (size_t)tiles * 8, stream), "alloc ranges");
    CS_TRY(pool_alloc(ctx, (void **)&s->n_last, pix_total * 4, stream), "alloc n_last");
    {
        // the state owns T_final (the backward needs it after the caller's buffers may be gone);
        // callers that asked for it get a copy once the blend has run
        CS_TRY(pool_alloc(ctx, (void **)&s->t_final_own, pix_total * 4, stream), "alloc t_final");
        s->user_t_final.assign(V, nullptr);
        size_t off = 0;
        for (int v = 0; v < V; ++v) {
            ViewDesc &vd = s->views[v];
            const size_t np = (size_t)vd.width * vd.height;
            vd.n_last = s->n_last + off;
            s->user_t_final[v] = vd.t_final;
            vd.t_final = s->t_final_own + off;
            off += np;
        }
    }
    CS_TRY(put_views(s->views_dev, s->views.data(), V, stream), "copy views");
    CS_TRY(pool_alloc(ctx, (void **)&total, sizeof(PreprocessStats), stream), "alloc");
    CS_TRY(fill_words(total, 0u, sizeof(PreprocessStats), stream), "clear totals");
    {
        StageTimer tm(ctx, CS_STAGE_PREPROCESS, stream);
        PreprocessOut po{s->records, s->depth_keys, s->rects, s->counts, s->bboxes, radii,
                         reinterpret_cast<uint32_t *>(radii + R), reinterpret_cast<PreprocessStats *>(total)};
        CS_TRY(launch_preprocess(s->views_dev, s->views.data(), V, max_n, s->k, s->st, po, stream), "preprocess");
    }
    {
        // the depth sort's buffers (sized by the records alone) are taken while the preprocess runs
        const size_t scan_words = scan_tmp_words(R > 256 * 8 ? R : 256 * 8) + scan_tmp_words(256 * ((R + 4095) / 4096 + 1));
        CS_TRY(pool_alloc(ctx, (void **)&sort_keys_a, (size_t)R * 4, stream), "alloc");
        CS_TRY(pool_alloc(ctx, (void **)&sort_keys_b, (size_t)R * 4, stream), "alloc");
        CS_TRY(pool_alloc(ctx, (void **)&sort_vals_a, (size_t)R * 4, stream), "alloc");
        CS_TRY(pool_alloc(ctx, (void **)&sort_vals_b, (size_t)R * 4, stream), "alloc");
        CS_TRY(pool_alloc(ctx, (void **)&offsets, (size_t)R * 4, stream), "alloc");
        CS_TRY(pool_alloc(ctx, (void **)&radix_tmp, radix_tmp_words(R) * 4, stream), "alloc");
        CS_TRY(pool_alloc(ctx, (void **)&scan_tmp, scan_words * 8, stream), "alloc");
    }
    // The forward's one host synchronisation: the pair count (to size the pair lists) and the range
    // of the drawn records' depth keys; the depth sort orders only the low bits in which they differ
    // (the drawn keys share the others; undrawn records emit no pairs).  Its first pass, on key bits
    // 0-7, needs neither, so it runs on the device while the host waits for the totals.
    CS_TRY(publish_words(total, ctx->host_total_dev, (int)(sizeof(PreprocessStats) / 4), stream), "read totals");
    CS_TRY(cudaEventRecord(ctx->totals_ready, stream), "record");
    if (R > 1) {
        StageTimer tm(ctx, CS_STAGE_DEPTH_SORT, stream);
        CS_TRY(radix_sort_pairs(sort_keys_a, sort_vals_a, sort_keys_b, sort_vals_b, R, 8, radix_tmp, scan_tmp, &in_b,
                                stream, s->depth_keys, 0u),
               "depth sort");
    }
    CS_TRY(cudaEventSynchronize(ctx->totals_ready), "synchronize");
    {
        const PreprocessStats tot = *reinterpret_cast<const PreprocessStats *>(ctx->host_total);
        P = tot.pairs;
        if (P >= 0xffffffffull) {
            st_code = fail(CS_ERR_ARG, "%llu tile pairs exceed the 32-bit pair index", (unsigned long long)P);
            goto cleanup;
        }
        const uint32_t differ = P ? (~tot.key_min_inv) ^ tot.key_max : 0u;
        depth_bits = differ ? 32 - __builtin_clz(differ) : 0;
    }
    // depth order of the records
    {
        {
            StageTimer tm(ctx, CS_STAGE_DEPTH_SORT, stream);
            if (R <= 1) {
                CS_TRY(launch_depth_sort_input(s->depth_keys, R, 0u, sort_keys_a, sort_vals_a, stream), "sort input");
            } else if (depth_bits > 8) {  // the remaining passes, bits 8 .. depth_bits - 1
                bool b2 = false;
                if (in_b) {
                    CS_TRY(radix_sort_pairs(sort_keys_b, sort_vals_b, sort_keys_a, sort_vals_a, R, depth_bits, radix_tmp,
                                            scan_tmp, &b2, stream, nullptr, 0u, 8, true),
                           "depth sort");
                    in_b = !b2;
                } else {
                    CS_TRY(radix_sort_pairs(sort_keys_a, sort_vals_a, sort_keys_b, sort_vals_b, R, depth_bits, radix_tmp,
                                            scan_tmp, &b2, stream, nullptr, 0u, 8, true),
                           "depth sort");
                    in_b = b2;
                }
            }
        }
        uint32_t *sorted = in_b ? sort_vals_b : sort_vals_a;
        if (V > 1) {
            // group the depth-ordered records view by view (stable): pairs are then emitted per view
            StageTimer tv(ctx, CS_STAGE_DEPTH_SORT, stream);
            uint32_t *vk = in_b ? sort_keys_b : sort_keys_a, *vk2 = in_b ? sort_keys_a : sort_keys_b;
            uint32_t *vv2 = in_b ? sort_vals_a : sort_vals_b;
            CS_TRY(launch_view_keys(s->views_dev, V, sorted, R, vk, stream, true), "view keys");
            bool vb = false;
            CS_TRY(radix_sort_pairs(vk, sorted, vk2, vv2, R, view_bits, radix_tmp, scan_tmp, &vb, stream, nullptr, 0u, 0,
                                    true),
                   "view sort");
            if (vb) sorted = vv2;
        }
        StageTimer tm(ctx, CS_STAGE_SCAN_EMIT, stream);
        // the depth (or view) sort's last kernel precedes it
        CS_TRY(launch_exclusive_scan(s->counts, sorted, offsets, R, nullptr, scan_tmp, stream, R > 0), "scan");
        s->n_pairs = (int64_t)P;
        CS_TRY(pool_alloc(ctx, (void **)&s->pair_keys, P * 4, stream), "alloc pairs");
        CS_TRY(pool_alloc(ctx, (void **)&s->pair_vals, P * 4, stream), "alloc pairs");
        CS_TRY(pool_alloc(ctx, (void **)&pk_b, P * 4, stream), "alloc pairs");
        CS_TRY(pool_alloc(ctx, (void **)&pv_b, P * 4, stream), "alloc pairs");
        CS_TRY(launch_emit_pairs(s->views_dev, V, sorted, offsets, s->counts, s->rects, s->records, radii,
                                 reinterpret_cast<const uint32_t *>(radii + R), s->bboxes,
                                 R, local_bits, s->mask_shift, s->pair_keys, s->pair_vals, stream, (uint32_t)P),
               "emit pairs");
        pool_free(radii, stream);
        radii = nullptr;
    }
    // stable sort of the pairs by tile
    {
        StageTimer tm(ctx, CS_STAGE_TILE_SORT, stream);
        pool_free(radix_tmp, stream);
        pool_free(scan_tmp, stream);
        radix_tmp = nullptr;
        scan_tmp = nullptr;
        const int64_t nbk = ((int64_t)P + 4095) / 4096;
        CS_TRY(pool_alloc(ctx, (void **)&radix_tmp, radix_tmp_words((int64_t)P) * 4, stream), "alloc");
        CS_TRY(pool_alloc(ctx, (void **)&scan_tmp, scan_tmp_words(256 * (nbk + 1)) * 8, stream), "alloc");
        CS_TRY(radix_sort_pairs(s->pair_keys, s->pair_vals, pk_b, pv_b, (int64_t)P, local_bits, radix_tmp, scan_tmp,
                                &in_b, stream),
               "tile sort");
        if (in_b) {
            uint32_t *t = s->pair_keys; s->pair_keys = pk_b; pk_b = t;
            t = s->pair_vals; s->pair_vals = pv_b; pv_b = t;
        }
        CS_TRY(launch_tile_ranges(s->pair_keys, (int64_t)P, s->views_dev, local_bits, s->mask_shift, s->ranges, tiles,
                                  stream, V),
               "tile ranges");
    }
    if (s->st.tile_split == 0 && (s->view_done.empty() || persist) && tiles > 0) {
        // the blends launch the tiles longest pair list first (both passes use the order); the
        // persistent launch of several views takes them view by view, and its counters (tile
        // queue, tiles done per view) follow the order, zeroed by the same kernel
        StageTimer tm(ctx, CS_STAGE_TILE_SORT, stream);
        const int n_zero = persist ? 1 + V : 0;
        CS_TRY(pool_alloc(ctx, (void **)&s->tile_order, ((size_t)tiles + n_zero) * 4, stream), "alloc");
        CS_TRY(launch_tile_order(s->ranges, tiles, s->tile_order, s->views_dev, V, persist, s->tile_order + tiles,
                                 n_zero, stream),
               "tile order");
    }
    if (s->st.tile_split > 0 && P > 0) {
        // tile split: which tiles are heavy, their chunk slots, the work items; the totals size the
        // items and the chunk states, so they are read back (a second host synchronisation)
        StageTimer tm(ctx, CS_STAGE_TILE_SORT, stream);
        const uint32_t split = (uint32_t)s->st.tile_split;
        uint32_t *heavy = nullptr, *light = nullptr, *heavy_base = nullptr, *light_base = nullptr;
        unsigned long long *tot = nullptr, *stmp = nullptr;
        unsigned int *cnt = nullptr;
        cudaError_t e = pool_alloc(ctx, (void **)&heavy, (size_t)tiles * 4, stream);
        if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&light, (size_t)tiles * 4, stream);
        if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&heavy_base, (size_t)tiles * 4, stream);
        if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&light_base, (size_t)tiles * 4, stream);
        if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&tot, 2 * sizeof(unsigned long long), stream);
        if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&cnt, 2 * sizeof(unsigned int), stream);
        if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&stmp, scan_tmp_words(tiles) * 8, stream);
        if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&s->split_slot, (size_t)tiles * 4, stream);
        if (e == cudaSuccess) e = fill_words(cnt, 0u, 2 * sizeof(unsigned int), stream);
        if (e == cudaSuccess) e = launch_split_count(s->ranges, tiles, split, heavy, light, cnt, stream);
        if (e == cudaSuccess) e = launch_exclusive_scan(heavy, nullptr, heavy_base, tiles, tot, stmp, stream);
        if (e == cudaSuccess) e = launch_exclusive_scan(light, nullptr, light_base, tiles, tot + 1, stmp, stream);
        if (e == cudaSuccess)
            e = publish_words(tot, ctx->host_total_dev, 4, stream);
        if (e == cudaSuccess)
            e = publish_words(cnt, ctx->host_total_dev + 2, 1, stream);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->totals_ready, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(ctx->totals_ready);
        uint64_t n_slots = 0, n_light = 0, n_heavy = 0;
        if (e == cudaSuccess) {
            n_slots = ctx->host_total[0];
            n_light = ctx->host_total[1];
            n_heavy = (uint64_t)(*reinterpret_cast<const unsigned int *>(ctx->host_total + 2));
            s->n_items = (uint32_t)(n_slots + n_light);
            s->n_heavy = (uint32_t)n_heavy;
            e = pool_alloc(ctx, (void **)&s->split_items, (size_t)s->n_items * sizeof(uint2), stream);
        }
        if (e == cudaSuccess) e = pool_alloc(ctx, (void **)&s->split_heavy, (size_t)(n_heavy + 1) * sizeof(uint2), stream);
        if (e == cudaSuccess)
            e = pool_alloc(ctx, (void **)&s->chunk_state, (size_t)(n_slots + 1) * SPLIT_STATE_FLOATS * 4, stream);
        if (e == cudaSuccess)
            e = launch_split_items(s->ranges, tiles, split, heavy_base, light_base, (uint32_t)n_slots, s->split_items,
                                   s->split_heavy, cnt + 1, s->split_slot, stream);
        pool_free(heavy, stream);
        pool_free(light, stream);
        pool_free(heavy_base, stream);
        pool_free(light_base, stream);
        pool_free(tot, stream);
        pool_free(cnt, stream);
        pool_free(stmp, stream);
        CS_TRY(e, "tile split plan");
    }
    {
        StageTimer tm(ctx, CS_STAGE_BLEND, stream);
        BlendArgs a{s->views_dev, V, s->ranges, s->pair_vals, s->records, s->bboxes, s->st, tiles, s->k,
                    s->pair_keys, s->mask_shift};
        a.n_pairs = (uint32_t)P;
        a.n_records = (uint32_t)R;
        set_split_args(a, s);
        if (persist && s->tile_order) {
            // one persistent launch over all views; each view's flag is raised when its last tile
            // is written (the events, recorded after the launch, mark the whole batch)
            a.queue = s->tile_order + tiles;
            a.view_tiles_done = s->tile_order + tiles + 1;
            a.view_flags = s->view_flags;
            a.flag_value = s->flag_value;
            CS_TRY(launch_blend_forward(a, stream), "blend");
            for (int v = 0; v < V; ++v) CS_TRY(cudaEventRecord(s->view_done[v], stream), "record view");
        } else if (s->view_done.size() == (size_t)V && !a.split) {
            for (int v = 0; v < V; ++v) {  // one launch per view, each view's completion recorded
                const ViewDesc &vd = s->views[v];
                BlendArgs av = a;
                av.tile_offset = vd.tile_base;
                av.n_tiles = (uint32_t)(vd.tiles_x * vd.tiles_y);
                CS_TRY(launch_blend_forward(av, stream), "blend");
                CS_TRY(cudaEventRecord(s->view_done[v], stream), "record view");
            }
        } else {
            CS_TRY(launch_blend_forward(a, stream), "blend");
            for (size_t v = 0; v < s->view_done.size(); ++v)  // every view is complete at once
                CS_TRY(cudaEventRecord(s->view_done[v], stream), "record view");
        }
    }
    for (int v = 0; v < V; ++v) {
        const ViewDesc &vd = s->views[v];
        if (s->user_t_final[v]) {
            CS_TRY(cudaMemcpyAsync(s->user_t_final[v], vd.t_final, (size_t)vd.width * vd.height * 4,
                                   cudaMemcpyDeviceToDevice, stream),
                   "copy t_final");
        }
    }
cleanup:
    pool_free(radii, stream);
    pool_free(sort_keys_a, stream);
    pool_free(sort_keys_b, stream);
    pool_free(sort_vals_a, stream);
    pool_free(sort_vals_b, stream);
    pool_free(offsets, stream);
    pool_free(radix_tmp, stream);
    pool_free(scan_tmp, stream);
    pool_free(total, stream);
    pool_free(pk_b, stream);
    pool_free(pv_b, stream);
    return st_code;
}

extern "C" cs_status cs_forward(cs_context *ctx, const cs_scene *scene, const cs_camera *cams, int32_t n_views,
                                const cs_settings *settings, float *image, float *t_final, cs_fwd_state **state_out,
                                void *stream_ptr) {
    if (state_out) *state_out = nullptr;
    if (!ctx) return fail(CS_ERR_ARG, "context is NULL");
    cs_status st;
    if ((st = check_scene(scene)) != CS_OK) return st;
    if ((st = check_settings(settings)) != CS_OK) return st;
    if (!cams || n_views <= 0 || n_views > 1024) return fail(CS_ERR_ARG, "need 1..1024 cameras");
    if (!image) return fail(CS_ERR_ARG, "image is NULL");
    for (int v = 0; v < n_views; ++v) {
        if ((st = check_camera(&cams[v])) != CS_OK) return st;
        if (cams[v].width != cams[0].width || cams[v].height != cams[0].height)
            return fail(CS_ERR_ARG, "cs_forward: all views must have the same size");
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    cs_fwd_state *s = new (std::nothrow) cs_fwd_state();
    if (!s) return fail(CS_ERR_NOMEM, "out of host memory");
    s->ctx = ctx;
    s->scene = *scene;
    s->k = scene->k;
    s->st = to_settings(*settings);
    s->settings = *settings;
    s->views.resize(n_views);
    const size_t hw = (size_t)cams[0].width * cams[0].height;
    for (int v = 0; v < n_views; ++v) {
        ViewDesc &vd = s->views[v];
        fill_view(vd, cams[v]);
        vd.points = scene->points; vd.delta = scene->delta; vd.sigma = scene->sigma;
        vd.opacity = scene->opacity; vd.sh = scene->sh;
        vd.n = scene->n; vd.k = scene->k; vd.sh_degree = scene->sh_degree; vd.activation = scene->activation; vd.storage = scene->storage;
        vd.image = image + (size_t)v * 3 * hw;
        vd.t_final = t_final ? t_final + (size_t)v * hw : nullptr;
    }
    st = run_forward(ctx, s, stream);
    if (st == CS_OK) st = take_device_status(stream, "cs_forward");
    if (st != CS_OK || !state_out) {
        state_free(s);
        return st;
    }
    *state_out = s;
    return CS_OK;
}

extern "C" cs_status cs_debug_set_pair_value(cs_fwd_state *s, int64_t index, uint32_t value) {
    if (!s) return fail(CS_ERR_ARG, "state is NULL");
#if CS_CHECKED
    if (index < 0 || index >= s->n_pairs) return fail(CS_ERR_ARG, "pair %lld outside 0..%lld", (long long)index,
                                                      (long long)s->n_pairs);
    DeviceGuard dg(s->ctx->device);
    cudaError_t e = cudaMemcpyAsync(s->pair_vals + index, &value, sizeof value, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return fail_cuda(e, "cs_debug_set_pair_value");
    return CS_OK;
#else
    (void)index;
    (void)value;
    return fail(CS_ERR_STATE, "cs_debug_set_pair_value: only in checked builds");
#endif
}

static cs_status run_backward(cs_context *ctx, const cs_fwd_state *s, const float *dL_dimage, float *dpoints,
                              float *ddelta, float *dsigma, float *dopacity, float *dsh, void *stream_ptr, bool write);

extern "C" cs_status cs_backward(cs_context *ctx, const cs_fwd_state *s, const float *dL_dimage, float *dpoints,
                                 float *ddelta, float *dsigma, float *dopacity, float *dsh, void *stream_ptr) {
    return run_backward(ctx, s, dL_dimage, dpoints, ddelta, dsigma, dopacity, dsh, stream_ptr, false);
}

extern "C" cs_status cs_backward_write(cs_context *ctx, const cs_fwd_state *s, const float *dL_dimage, float *dpoints,
                                       float *ddelta, float *dsigma, float *dopacity, float *dsh, void *stream_ptr) {
    return run_backward(ctx, s, dL_dimage, dpoints, ddelta, dsigma, dopacity, dsh, stream_ptr, true);
}

static cs_status run_backward(cs_context *ctx, const cs_fwd_state *s, const float *dL_dimage, float *dpoints,
                              float *ddelta, float *dsigma, float *dopacity, float *dsh, void *stream_ptr, bool write) {
    if (!ctx || !s) return fail(CS_ERR_ARG, "context or state is NULL");
    if (s->ctx != ctx) return fail(CS_ERR_STATE, "state belongs to another context");
    if (!dL_dimage) return fail(CS_ERR_ARG, "dL_dimage is NULL");
    if (s->settings.alpha_max > 0.999f)
        return fail(CS_ERR_ARG, "the backward needs alpha_max <= 0.999 (T is recovered by dividing by 1 - alpha)");
    DeviceGuard dg(ctx->device);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    const int V = (int)s->views.size();
    cs_status st_code = CS_OK;
    float4 *grads = nullptr;
    if (write && (V > 1 || s->n_records == 0)) {
        // several views add into shared gradients with atomics: clear them first
        const int64_t n = s->scene.n;
        const int64_t nb = (int64_t)(s->scene.sh_degree + 1) * (s->scene.sh_degree + 1);
        cudaError_t e = cudaSuccess;
        if (dpoints) e = fill_words(dpoints, 0u, (size_t)n * s->k * 3 * 4, stream);
        if (e == cudaSuccess && ddelta) e = fill_words(ddelta, 0u, (size_t)n * 4, stream);
        if (e == cudaSuccess && dsigma) e = fill_words(dsigma, 0u, (size_t)n * 4, stream);
        if (e == cudaSuccess && dopacity) e = fill_words(dopacity, 0u, (size_t)n * 4, stream);
        if (e == cudaSuccess && dsh) e = fill_words(dsh, 0u, (size_t)(n * nb * 3) * 4, stream);
        if (e != cudaSuccess) return fail_cuda(e, "clear gradients");
    }
    if (s->n_records == 0) return CS_OK;
    {
        cudaError_t e = pool_alloc(ctx, (void **)&grads, (size_t)s->n_records * GRAD_WORDS * 4, stream);
        if (e != cudaSuccess) return fail_cuda(e, "alloc gradient records");
        e = fill_words(grads, 0u, (size_t)s->n_records * GRAD_WORDS * 4, stream);
        if (e == cudaSuccess) {
            StageTimer tm(ctx, CS_STAGE_BLEND_BACKWARD, stream);
            BlendArgs a{s->views_dev, V, s->ranges, s->pair_vals, s->records, s->bboxes, s->st, s->n_tiles, s->k,
                        s->pair_keys, s->mask_shift};
            a.n_pairs = (uint32_t)s->n_pairs;
            a.n_records = (uint32_t)s->n_records;
            set_split_args(a, s);
            const int64_t stride = (int64_t)3 * s->views[0].width * s->views[0].height;
            e = launch_blend_backward(a, dL_dimage, stride, grads, stream);
        }
        if (e == cudaSuccess) {
            StageTimer tm(ctx, CS_STAGE_PREPROCESS_BACKWARD, stream);
            PreprocessGrads g{dpoints, ddelta, dsigma, dopacity, dsh};
            g.write = write && V == 1;
            e = launch_preprocess_backward(s->views_dev, V, s->scene.n, s->k, s->scene.sh_degree, s->scene.storage,
                                           s->st, s->records, s->counts, grads, g, V > 1, stream);
        }
        if (e != cudaSuccess) st_code = fail_cuda(e, "backward");
    }
    pool_free(grads, stream);
    if (st_code == CS_OK) st_code = take_device_status(stream, "cs_backward");
    return st_code;
}

extern "C" void cs_state_release(cs_fwd_state *s) { state_free(s); }

extern "C" cs_status cs_state_sizes(const cs_fwd_state *s, int64_t *records, int64_t *pairs, int64_t *tiles) {
    if (!s) return fail(CS_ERR_ARG, "state is NULL");
    if (records) *records = s->n_records;
    if (pairs) *pairs = s->n_pairs;
    if (tiles) *tiles = s->n_tiles;
    return CS_OK;
}

extern "C" cs_status cs_state_copy(const cs_fwd_state *s, int32_t which, void *host_dst, size_t capacity,
                                   size_t *bytes_out) {
    if (!s) return fail(CS_ERR_ARG, "state is NULL");
    const void *src = nullptr;
    size_t bytes = 0;
    size_t pix = 0;
    for (const ViewDesc &vd : s->views) pix += (size_t)vd.width * vd.height;
    switch (which) {
        case CS_ARR_RECORDS: src = s->records; bytes = (size_t)s->n_records * REC_WORDS * 4; break;
        case CS_ARR_DEPTH_KEYS: src = s->depth_keys; bytes = (size_t)s->n_records * 4; break;
        case CS_ARR_RECTS: src = s->rects; bytes = (size_t)s->n_records * 8; break;
        case CS_ARR_COUNTS: src = s->counts; bytes = (size_t)s->n_records * 4; break;
        case CS_ARR_PAIR_KEYS: src = s->pair_keys; bytes = (size_t)s->n_pairs * 4; break;
        case CS_ARR_PAIR_VALUES: src = s->pair_vals; bytes = (size_t)s->n_pairs * 4; break;
        case CS_ARR_TILE_RANGES: src = s->ranges; bytes = (size_t)s->n_tiles * 8; break;
        case CS_ARR_N_LAST: src = s->n_last; bytes = pix * 4; break;
        case CS_ARR_HULLS: break;
        case CS_ARR_TILE_ORDER: src = s->tile_order; bytes = s->tile_order ? (size_t)s->n_tiles * 4 : 0; break;
        default: return fail(CS_ERR_ARG, "unknown array %d", which);
    }
    if (which == CS_ARR_HULLS) bytes = (size_t)s->n_records * 4;
    if (bytes_out) *bytes_out = bytes;
    if (!host_dst) return CS_OK;
    if (capacity < bytes) return fail(CS_ERR_ARG, "capacity %zu < %zu bytes", capacity, bytes);
    DeviceGuard dg(s->ctx->device);
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return fail_cuda(e, "synchronize");
    if (which == CS_ARR_HULLS) {
        // word 7 of every record; records that are not drawn report 0
        std::vector<uint32_t> rec((size_t)s->n_records * REC_WORDS), cnt((size_t)s->n_records);
        if (s->n_records) {
            e = cudaMemcpy(rec.data(), s->records, rec.size() * 4, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemcpy(cnt.data(), s->counts, cnt.size() * 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return fail_cuda(e, "copy");
        }
        uint32_t *d = (uint32_t *)host_dst;
        for (int64_t r = 0; r < s->n_records; ++r) d[r] = cnt[r] ? rec[(size_t)r * REC_WORDS + R_HULL] : 0u;
        return CS_OK;
    }
    if (bytes) {
        e = cudaMemcpy(host_dst, src, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail_cuda(e, "copy");
    }
    if (which == CS_ARR_PAIR_KEYS && s->mask_shift) {  // the documented layout: block masks removed
        uint32_t *d = (uint32_t *)host_dst;
        const uint32_t keep = (1u << s->mask_shift) - 1u;
        for (int64_t q = 0; q < s->n_pairs; ++q) d[q] &= keep;
    }
    return CS_OK;
}

// ---------------------------------------------------------------------------------------------
// host-buffer step and work counters
// ---------------------------------------------------------------------------------------------
// the device address of host buffer p when kernels on `device` can read and write it in place:
// pinned or registered memory, or any host memory where the GPU walks the host's page tables
// (on a Grace host, over NVLink-C2C); NULL otherwise
static void *device_view(const void *p, int device) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged)
        return a.devicePointer ? a.devicePointer : const_cast<void *>(p);
    if (a.type == cudaMemoryTypeUnregistered) {
        int pageable = 0;
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccessUsesHostPageTables, device);
        if (pageable) return const_cast<void *>(p);
    }
    return nullptr;
}

extern "C" cs_status cs_step_host(cs_context *ctx, const cs_scene *sh, const cs_camera *cams, int32_t n_views,
                                  const cs_settings *settings, const float *dL_host, float *image_host,
                                  float *dpoints_host, float *ddelta_host, float *dsigma_host, float *dopacity_host,
                                  float *dsh_host, void *stream_ptr) {
    if (!ctx) return fail(CS_ERR_ARG, "context is NULL");
    cs_status st;
    if ((st = check_scene(sh)) != CS_OK) return st;
    if (!cams || n_views <= 0 || !image_host) return fail(CS_ERR_ARG, "cameras and image are required");
    DeviceGuard dg(ctx->device);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    const int64_t n = sh->n;
    const int nb = (sh->sh_degree + 1) * (sh->sh_degree + 1);
    const size_t esz = sh->storage == CS_STORE_F32 ? 4 : 2;  // parameters as stored; gradients float32
    const size_t b_pts = (size_t)n * sh->k * 3, b_one = (size_t)n, b_sh = (size_t)n * nb * 3;
    const size_t b_img = (size_t)n_views * 3 * cams[0].width * cams[0].height * 4;
    const bool bwd = dL_host != nullptr;
    // The scene is copied to the device (the preprocess stages it with cp.async).  dL/dimage, the
    // image and, with one view, the gradients are read and written in place by the kernels when
    // the device can reach the host buffers, so the gradients stream out while the preprocess
    // backward computes them; otherwise they go through device buffers and copies.
    float *outs_host[5] = {dpoints_host, ddelta_host, dsigma_host, dopacity_host, dsh_host};
    float *dl_view = bwd ? static_cast<float *>(device_view(dL_host, ctx->device)) : nullptr;
    float *img_view = static_cast<float *>(device_view(image_host, ctx->device));
    float *g_view[5] = {};
    bool grads_direct = bwd && n_views == 1;
    for (int i = 0; i < 5; ++i) {
        g_view[i] = static_cast<float *>(device_view(outs_host[i], ctx->device));
        if (outs_host[i] && !g_view[i]) grads_direct = false;
    }
    float *d[12] = {};
    const size_t sizes[12] = {b_pts * esz, b_one * esz, b_one * esz, b_one * esz, b_sh * esz, b_img,
                              b_img,       b_pts * 4,   b_one * 4,   b_one * 4,   b_one * 4, b_sh * 4};
    bool need[12] = {true, true, true, true, true, !img_view, bwd && !dl_view};
    for (int i = 7; i < 12; ++i) need[i] = bwd && !grads_direct;
    cs_fwd_state *state = nullptr;
    cs_status code = CS_OK;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 12 && e == cudaSuccess; ++i)
        if (need[i]) e = pool_alloc(ctx, (void **)&d[i], sizes[i], stream);
    const void *srcs[5] = {sh->points, sh->delta, sh->sigma, sh->opacity, sh->sh};
    for (int i = 0; i < 5 && e == cudaSuccess; ++i)
        if (sizes[i]) e = cudaMemcpyAsync(d[i], srcs[i], sizes[i], cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && need[6]) e = cudaMemcpyAsync(d[6], dL_host, b_img, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) code = fail_cuda(e, "cs_step_host upload");
    float *img = img_view ? img_view : d[5];
    const float *dl = dl_view ? dl_view : d[6];
    float *gout[5];
    for (int i = 0; i < 5; ++i) gout[i] = grads_direct ? g_view[i] : (outs_host[i] ? d[7 + i] : nullptr);
    if (code == CS_OK) {
        cs_scene dev = *sh;
        dev.points = d[0]; dev.delta = d[1]; dev.sigma = d[2]; dev.opacity = d[3]; dev.sh = d[4];
        code = cs_forward(ctx, &dev, cams, n_views, settings, img, nullptr, bwd ? &state : nullptr, stream_ptr);
        if (code == CS_OK && bwd)
            code = cs_backward_write(ctx, state, dl, gout[0], gout[1], gout[2], gout[3], gout[4], stream_ptr);
    }
    if (code == CS_OK) {
        if (!img_view) e = cudaMemcpyAsync(image_host, d[5], b_img, cudaMemcpyDeviceToHost, stream);
        for (int i = 0; i < 5 && e == cudaSuccess && bwd && !grads_direct; ++i)
            if (outs_host[i] && sizes[7 + i])
                e = cudaMemcpyAsync(outs_host[i], d[7 + i], sizes[7 + i], cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) code = fail_cuda(e, "cs_step_host download");
    }
    if (state) state_free(state);
    for (int i = 0; i < 12; ++i) pool_free(d[i], stream);
    return code;
}

// The worker thread of the pipelined host-buffer steps: takes the queued steps in ticket order and
// enqueues, for each, the forward and backward on the compute stream (after its upload, and after
// the slot's previous outputs have been copied out) and the copies of its outputs on the download
// stream.  The forward's pair-count readback blocks this thread, not the caller's.
static void host_worker_loop(cs_context *ctx) {
    cudaSetDevice(ctx->device);
    for (;;) {
        cs_context::HostJob job;
        {
            std::unique_lock<std::mutex> lk(ctx->job_mu);
            ctx->job_cv.wait(lk, [&] { return ctx->worker_stop || !ctx->jobs.empty(); });
            if (ctx->jobs.empty()) return;  // stopping, nothing left
            job = ctx->jobs.front();
            ctx->jobs.pop_front();
        }
        cs_context::HostSlot &sl = ctx->host_slots[job.slot];
        cs_status code = CS_OK;
        cudaError_t e = cudaStreamWaitEvent(ctx->compute_stream, sl.uploaded, 0);
        // the slot's previous step (ticket - HOST_SLOTS), if any, was enqueued before this one:
        // its outputs must be copied out before this step writes over them
        if (e == cudaSuccess && job.ticket > (uint64_t)cs_context::HOST_SLOTS)
            e = cudaStreamWaitEvent(ctx->compute_stream, sl.done, 0);
        if (e != cudaSuccess) code = fail_cuda(e, "cs_step_host_submit: stream order");
        float *g[5];
        for (int i = 0; i < 5; ++i)
            g[i] = job.bwd && job.outs_host[i] ? static_cast<float *>(job.d[7 + i]) : nullptr;
        cs_fwd_state *state = nullptr;
        if (code == CS_OK)
            code = cs_forward(ctx, &job.scene, &job.cam, 1, job.has_settings ? &job.settings : nullptr,
                              static_cast<float *>(job.d[6]), nullptr, job.bwd ? &state : nullptr,
                              ctx->compute_stream);
        if (code == CS_OK && job.bwd)
            code = cs_backward_write(ctx, state, static_cast<const float *>(job.d[5]), g[0], g[1], g[2], g[3], g[4],
                                     ctx->compute_stream);
        if (state) state_free(state);
        // recorded whatever happened above, so that no later wait waits on an older step
        e = cudaEventRecord(sl.computed, ctx->compute_stream);
        cudaError_t e2 = cudaStreamWaitEvent(ctx->download_stream, sl.computed, 0);
        if (e2 == cudaSuccess && code == CS_OK)
            e2 = cudaMemcpyAsync(job.image_host, job.d[6], job.sizes[6], cudaMemcpyDeviceToHost, ctx->download_stream);
        for (int i = 0; i < 5 && e2 == cudaSuccess && code == CS_OK; ++i)
            if (g[i] && job.sizes[7 + i])
                e2 = cudaMemcpyAsync(job.outs_host[i], g[i], job.sizes[7 + i], cudaMemcpyDeviceToHost,
                                     ctx->download_stream);
        const cudaError_t e3 = cudaEventRecord(sl.done, ctx->download_stream);
        if (code == CS_OK && e != cudaSuccess) code = fail_cuda(e, "cs_step_host_submit");
        if (code == CS_OK && e2 != cudaSuccess) code = fail_cuda(e2, "cs_step_host_submit: download");
        if (code == CS_OK && e3 != cudaSuccess) code = fail_cuda(e3, "cs_step_host_submit");
        {
            std::lock_guard<std::mutex> lk(ctx->job_mu);
            if (code != CS_OK && ctx->host_code == CS_OK) {
                ctx->host_code = code;
                ctx->host_msg = cs_last_error();
            }
            ctx->jobs_enqueued = job.ticket;
        }
        ctx->job_cv.notify_all();
    }
}

// blocks until the worker has enqueued the GPU work of every step up to `ticket`
static void wait_enqueued(cs_context *ctx, uint64_t ticket) {
    std::unique_lock<std::mutex> lk(ctx->job_mu);
    ctx->job_cv.wait(lk, [&] { return ctx->jobs_enqueued >= ticket; });
}

extern "C" cs_status cs_step_host_submit(cs_context *ctx, const cs_scene *sh, const cs_camera *cam,
                                         const cs_settings *settings, const float *dL_host, float *image_host,
                                         float *dpoints_host, float *ddelta_host, float *dsigma_host,
                                         float *dopacity_host, float *dsh_host, uint64_t *ticket) {
    if (!ctx || !ticket) return fail(CS_ERR_ARG, "cs_step_host_submit: context and ticket are required");
    cs_status st;
    if ((st = check_scene(sh)) != CS_OK) return st;
    if (!cam || !image_host) return fail(CS_ERR_ARG, "cs_step_host_submit: camera and image are required");
    if ((st = check_camera(cam)) != CS_OK) return st;
    if (settings && (st = check_settings(settings)) != CS_OK) return st;
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->host_mu);
    const bool bwd = dL_host != nullptr;
    cudaError_t e = cudaSuccess;
    if (!ctx->upload_stream) {  // streams and events, each created once (kept if a later one fails)
        if (!ctx->compute_stream) e = cudaStreamCreateWithFlags(&ctx->compute_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess && !ctx->download_stream)
            e = cudaStreamCreateWithFlags(&ctx->download_stream, cudaStreamNonBlocking);
        for (auto &sl : ctx->host_slots) {
            if (e == cudaSuccess && !sl.uploaded) e = cudaEventCreateWithFlags(&sl.uploaded, cudaEventDisableTiming);
            if (e == cudaSuccess && !sl.computed) e = cudaEventCreateWithFlags(&sl.computed, cudaEventDisableTiming);
            if (e == cudaSuccess && !sl.done) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        }
        // the upload stream last: once it exists, everything else does
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->upload_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail_cuda(e, "cs_step_host_submit: streams and events");
    }
    if (!ctx->host_worker.joinable()) {  // started with the first step (again if that failed)
        try {
            ctx->host_worker = std::thread(host_worker_loop, ctx);
        } catch (...) {
            return fail(CS_ERR_CUDA, "cs_step_host_submit: cannot start the worker thread");
        }
    }
    const uint64_t t = ctx->host_tickets + 1;
    const int slot = (int)(t % cs_context::HOST_SLOTS);
    cs_context::HostSlot &sl = ctx->host_slots[slot];
    // the slot's previous step must have its GPU work enqueued (its events recorded) before this
    // step's copies are ordered after them
    if (sl.ticket) wait_enqueued(ctx, sl.ticket);
    cs_context::HostJob job;
    job.ticket = t;
    job.slot = slot;
    job.bwd = bwd;
    job.cam = *cam;
    job.has_settings = settings != nullptr;
    if (settings) job.settings = *settings;
    job.image_host = image_host;
    float *outs_host[5] = {dpoints_host, ddelta_host, dsigma_host, dopacity_host, dsh_host};
    for (int i = 0; i < 5; ++i) job.outs_host[i] = outs_host[i];
    // the slot's arrays: 0-4 scene (as stored), 5 dL/dimage, 6 image, 7-11 gradients (binary32)
    const int64_t n = sh->n;
    const int nb = (sh->sh_degree + 1) * (sh->sh_degree + 1);
    const size_t esz = sh->storage == CS_STORE_F32 ? 4 : 2;
    const size_t e_pts = (size_t)n * sh->k * 3, e_one = (size_t)n, e_sh = (size_t)n * nb * 3;
    const size_t b_img = (size_t)3 * cam->width * cam->height * 4;
    const size_t sizes[12] = {e_pts * esz, e_one * esz, e_one * esz, e_one * esz, e_sh * esz, bwd ? b_img : 0,
                              b_img,       e_pts * 4,   e_one * 4,   e_one * 4,   e_one * 4, e_sh * 4};
    size_t offs[12], total = 0;
    for (int i = 0; i < 12; ++i) {
        offs[i] = total;
        job.sizes[i] = sizes[i];
        const bool used = i < 7 || (bwd && outs_host[i - 7]);
        total += used ? (sizes[i] + 255) & ~(size_t)255 : 0;
    }
    if (sl.cap < total) {  // the slot's last step must be done with its buffers before they are replaced
        if (sl.ticket) e = cudaEventSynchronize(sl.done);
        if (sl.buf) cudaFree(sl.buf);
        sl.buf = nullptr;
        sl.cap = 0;
        if (e == cudaSuccess) e = cudaMalloc(&sl.buf, total);
        if (e != cudaSuccess) return fail_cuda(e, "cs_step_host_submit: slot buffers");
        sl.cap = total;
    }
    for (int i = 0; i < 12; ++i) job.d[i] = static_cast<char *>(sl.buf) + offs[i];
    // inputs: the copy into this slot waits (on the GPU) until the slot's previous step has read them
    if (sl.ticket) e = cudaStreamWaitEvent(ctx->upload_stream, sl.computed, 0);
    const void *srcs[6] = {sh->points, sh->delta, sh->sigma, sh->opacity, sh->sh, dL_host};
    for (int i = 0; i < 6 && e == cudaSuccess; ++i)
        if (sizes[i]) e = cudaMemcpyAsync(job.d[i], srcs[i], sizes[i], cudaMemcpyHostToDevice, ctx->upload_stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.uploaded, ctx->upload_stream);
    if (e != cudaSuccess) return fail_cuda(e, "cs_step_host_submit: upload");
    job.scene = *sh;
    job.scene.points = static_cast<float *>(job.d[0]);
    job.scene.delta = static_cast<float *>(job.d[1]);
    job.scene.sigma = static_cast<float *>(job.d[2]);
    job.scene.opacity = static_cast<float *>(job.d[3]);
    job.scene.sh = static_cast<float *>(job.d[4]);
    sl.ticket = t;
    ctx->host_tickets = t;
    {
        std::lock_guard<std::mutex> jl(ctx->job_mu);
        ctx->jobs.push_back(job);
    }
    ctx->job_cv.notify_all();
    *ticket = t;
    return CS_OK;
}

extern "C" cs_status cs_step_host_wait(cs_context *ctx, uint64_t ticket) {
    if (!ctx) return fail(CS_ERR_ARG, "context is NULL");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::mutex> lk(ctx->host_mu);
    if (ticket == 0 || ticket > ctx->host_tickets)
        return fail(CS_ERR_ARG, "cs_step_host_wait: ticket %llu was not submitted", (unsigned long long)ticket);
    wait_enqueued(ctx, ticket);
    // steps are copied out in order on the download stream, and the step last recorded in the
    // ticket's slot is this one or a later one
    const cudaError_t e = cudaEventSynchronize(ctx->host_slots[ticket % cs_context::HOST_SLOTS].done);
    {
        std::lock_guard<std::mutex> jl(ctx->job_mu);
        if (ctx->host_code != CS_OK) {  // reported once, with the worker's message
            const cs_status code = ctx->host_code;
            ctx->host_code = CS_OK;
            return fail(code, "%s", ctx->host_msg.c_str());
        }
    }
    if (e != cudaSuccess) return fail_cuda(e, "cs_step_host_wait");
    return take_device_status(ctx->compute_stream, "cs_step_host_wait");
}

extern "C" cs_status cs_work_counts(cs_context *ctx, const cs_fwd_state *s, const float *dL_dimage, uint64_t *counts,
                                    void *stream_ptr) {
    if (!ctx || !s || !counts) return fail(CS_ERR_ARG, "context, state and counts are required");
    DeviceGuard dg(ctx->device);
    cudaStream_t stream = (cudaStream_t)stream_ptr;
    unsigned long long *dc = nullptr;
    float4 *grads = nullptr;
    cudaError_t e = pool_alloc(ctx, (void **)&dc, 12 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, 12 * sizeof(unsigned long long), stream);
    const int V = (int)s->views.size();
    BlendArgs a{s->views_dev, V, s->ranges, s->pair_vals, s->records, s->bboxes, s->st, s->n_tiles, s->k,
                        s->pair_keys, s->mask_shift};
    a.n_pairs = (uint32_t)s->n_pairs;
    a.n_records = (uint32_t)s->n_records;
    if (e == cudaSuccess) e = launch_blend_forward(a, stream, dc);
    if (e == cudaSuccess && dL_dimage && s->n_records) {
        e = pool_alloc(ctx, (void **)&grads, (size_t)s->n_records * GRAD_WORDS * 4, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(grads, 0, (size_t)s->n_records * GRAD_WORDS * 4, stream);
        const int64_t stride = (int64_t)3 * s->views[0].width * s->views[0].height;
        if (e == cudaSuccess) e = launch_blend_backward(a, dL_dimage, stride, grads, stream, dc + 6);
    }
    unsigned long long host[12] = {};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, dc, sizeof host, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    pool_free(grads, stream);
    pool_free(dc, stream);
    if (e != cudaSuccess) return fail_cuda(e, "cs_work_counts");
    for (int i = 0; i < 12; ++i) counts[i] = host[i];
    return CS_OK;
}
