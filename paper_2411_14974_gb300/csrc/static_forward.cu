// Forward render that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they render: a host engine that
// owns every byte of device memory through its own arena (a hidden cudaMalloc would bypass its
// accounting and fragment its heap), a real-time loop that must not call into the driver's
// allocator (allocation can block or synchronise), or a plugin that is only allowed to allocate
// during its set-up phase.  For them cs_forward_static renders one view with every transient
// buffer carved out of one file-scope device array of fixed size; the caller passes only the
// scene, the camera and the output buffers.
//
// The array belongs to the library: every GPU that loads it holds the array until the process
// exits.  All calls share it and it keeps the last call's contents, so everything that must
// start at zero is cleared on the stream by each call, and calls that overlap on the GPU (two
// streams, two threads) race on it.  The first call on a device looks up the array's device
// address (cudaGetSymbolAddress) with that device current; make that first call before any
// stream capture.
#include <mutex>

#include "cs_api_internal.h"
#include "cs_common.cuh"

using namespace cs;

namespace {

constexpr size_t STATIC_BYTES = CS_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_BYTES];

std::mutex g_static_mu;
constexpr int MAX_DEVICES = 64;
unsigned char *g_static_addr[MAX_DEVICES] = {};

// bump carve-out of the static array, 256-byte aligned
struct Carve {
    unsigned char *base;
    size_t used = 0;
    template <class T>
    T *take(size_t count) {
        T *p = reinterpret_cast<T *>(base + used);
        used += (count * sizeof(T) + 255) & ~(size_t)255;
        return p;
    }
};

int bits_for(uint64_t n) {
    int b = 0;
    while (b < 32 && ((uint64_t)1 << b) < n) ++b;
    return b;
}

}  // namespace

extern "C" cs_status cs_forward_static(const cs_scene *scene, const cs_camera *cam, const cs_settings *settings,
                                       float *image, float *t_final, void *stream_ptr) {
    cs_status st;
    if ((st = check_scene(scene)) != CS_OK) return st;
    if ((st = check_settings(settings)) != CS_OK) return st;
    if (!cam || !image || !t_final) return fail(CS_ERR_ARG, "cs_forward_static: camera, image and t_final are required");
    if ((st = check_camera(cam)) != CS_OK) return st;
    if (scene->n > CS_STATIC_MAX_CONVEXES)
        return fail(CS_ERR_BUDGET, "cs_forward_static: %lld convexes exceed the static limit of %d",
                    (long long)scene->n, CS_STATIC_MAX_CONVEXES);
    if ((int64_t)cam->width * cam->height > CS_STATIC_MAX_PIXELS)
        return fail(CS_ERR_BUDGET, "cs_forward_static: %dx%d pixels exceed the static limit of %d", cam->width,
                    cam->height, CS_STATIC_MAX_PIXELS);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return fail(CS_ERR_ARG, "device %d out of range", dev);
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major * 10 + minor != 103) return fail(CS_ERR_CUDA, "device %d is sm_%d%d; built for sm_103a", dev, major, minor);
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (!g_static_addr[dev]) {
            // host code only holds a stand-in for the array; its device address comes from the runtime
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(static scratch)");
            g_static_addr[dev] = static_cast<unsigned char *>(p);
        }
        scratch = g_static_addr[dev];
    }
    cudaStream_t stream = (cudaStream_t)stream_ptr;

    ViewDesc vd;
    fill_view(vd, *cam);
    vd.points = scene->points; vd.delta = scene->delta; vd.sigma = scene->sigma;
    vd.opacity = scene->opacity; vd.sh = scene->sh;
    vd.n = scene->n; vd.k = scene->k; vd.sh_degree = scene->sh_degree; vd.activation = scene->activation; vd.storage = scene->storage;
    vd.image = image;
    vd.t_final = t_final;
    vd.rec_base = 0;
    vd.tile_base = 0;
    const int64_t R = scene->n;
    const uint32_t tiles = (uint32_t)(vd.tiles_x * vd.tiles_y);
    const size_t pixels = (size_t)cam->width * cam->height;
    const Settings s = to_settings(*settings);

    Carve c{scratch};
    ViewDesc *views_dev = c.take<ViewDesc>(1);
    float4 *records = c.take<float4>((size_t)CS_STATIC_MAX_CONVEXES * (REC_WORDS / 4));
    uint32_t *depth_keys = c.take<uint32_t>(CS_STATIC_MAX_CONVEXES);
    uint2 *rects = c.take<uint2>(CS_STATIC_MAX_CONVEXES);
    uint32_t *counts = c.take<uint32_t>(CS_STATIC_MAX_CONVEXES);
    float4 *bboxes = c.take<float4>(CS_STATIC_MAX_CONVEXES);
    float *radii = c.take<float>(CS_STATIC_MAX_CONVEXES);
    uint32_t *kept = c.take<uint32_t>(CS_STATIC_MAX_CONVEXES);
    uint32_t *ka = c.take<uint32_t>(CS_STATIC_MAX_CONVEXES), *kb = c.take<uint32_t>(CS_STATIC_MAX_CONVEXES);
    uint32_t *va = c.take<uint32_t>(CS_STATIC_MAX_CONVEXES), *vb = c.take<uint32_t>(CS_STATIC_MAX_CONVEXES);
    uint32_t *offsets = c.take<uint32_t>(CS_STATIC_MAX_CONVEXES);
    uint32_t *pk = c.take<uint32_t>(CS_STATIC_MAX_PAIRS), *pv = c.take<uint32_t>(CS_STATIC_MAX_PAIRS);
    uint32_t *pk2 = c.take<uint32_t>(CS_STATIC_MAX_PAIRS), *pv2 = c.take<uint32_t>(CS_STATIC_MAX_PAIRS);
    const int64_t max_sort = CS_STATIC_MAX_PAIRS > CS_STATIC_MAX_CONVEXES ? CS_STATIC_MAX_PAIRS : CS_STATIC_MAX_CONVEXES;
    uint32_t *radix_tmp = c.take<uint32_t>(radix_tmp_words(max_sort));
    unsigned long long *scan_tmp = c.take<unsigned long long>(scan_tmp_words(max_sort) + scan_tmp_words(256 * (max_sort / 4096 + 2)));
    PreprocessStats *totals = c.take<PreprocessStats>(1);
    uint2 *ranges = c.take<uint2>(tiles);
    uint32_t *n_last = c.take<uint32_t>(pixels);
    if (c.used > STATIC_BYTES) return fail(CS_ERR_BUDGET, "cs_forward_static: %dx%d needs more than the static array",
                                          cam->width, cam->height);
    vd.n_last = n_last;

    e = cudaMemcpyAsync(views_dev, &vd, sizeof vd, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(totals, 0, sizeof(PreprocessStats), stream);
    if (e == cudaSuccess) {
        PreprocessOut po{records, depth_keys, rects, counts, bboxes, radii, kept, totals};
        e = launch_preprocess(views_dev, &vd, 1, R, scene->k, s, po, stream);
    }
    // one host synchronisation: the pair count and the drawn records' depth-key range
    PreprocessStats tot{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, totals, sizeof tot, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail_cuda(e, "cs_forward_static");
    const unsigned long long P = tot.pairs;
    if (P > (unsigned long long)CS_STATIC_MAX_PAIRS)
        return fail(CS_ERR_BUDGET, "cs_forward_static: %llu tile pairs exceed the static limit of %d", P,
                    CS_STATIC_MAX_PAIRS);
    const uint32_t key_min = ~tot.key_min_inv;
    const int depth_bits = P ? bits_for((uint64_t)(tot.key_max - key_min) + 1) : 0;
    bool in_b = false;
    if (depth_bits > 0 && R > 1)  // the first pass reads the keys rebased, values = indices
        e = radix_sort_pairs(ka, va, kb, vb, R, depth_bits, radix_tmp, scan_tmp, &in_b, stream, depth_keys, key_min);
    else
        e = launch_depth_sort_input(depth_keys, R, key_min, ka, va, stream);
    const uint32_t *sorted = in_b ? vb : va;
    if (e == cudaSuccess) e = launch_exclusive_scan(counts, sorted, offsets, R, nullptr, scan_tmp, stream);
    const int local_bits = bits_for(tiles);
    const int mask_shift = local_bits + BLOCK_MASK_BITS <= 32 ? local_bits : 0;
    if (e == cudaSuccess)
        e = launch_emit_pairs(views_dev, 1, sorted, offsets, counts, rects, records, radii, kept, bboxes, R, local_bits,
                              mask_shift, pk, pv, stream, (uint32_t)P);
    if (e == cudaSuccess) e = radix_sort_pairs(pk, pv, pk2, pv2, (int64_t)P, local_bits, radix_tmp, scan_tmp, &in_b,
                                               stream);
    const uint32_t *keys = in_b ? pk2 : pk;
    const uint32_t *vals = in_b ? pv2 : pv;
    if (e == cudaSuccess)
        e = launch_tile_ranges(keys, (int64_t)P, views_dev, local_bits, mask_shift, ranges, tiles, stream, 1);
    if (e == cudaSuccess) {
        BlendArgs a{views_dev, 1, ranges, vals, records, bboxes, s, tiles, scene->k, keys, mask_shift};
        a.n_pairs = (uint32_t)P;
        a.n_records = (uint32_t)R;
        e = launch_blend_forward(a, stream);
    }
    if (e != cudaSuccess) return fail_cuda(e, "cs_forward_static");
    return take_device_status(stream, "cs_forward_static");
}
