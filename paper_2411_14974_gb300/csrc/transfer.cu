// Small device-side transfers of the forward and backward: buffer fills, the upload of the view
// descriptors and the publication of the forward's totals to mapped host memory.  They are kernels
// rather than cudaMemsetAsync / cudaMemcpyAsync so that nothing on the compute stream waits in a
// copy engine's queue: while pipelined host-buffer steps run, the copy engines carry hundreds of
// megabytes of scene upload and gradient download per step, and a copy queued behind one of
// those transfers would hold the compute stream for its whole duration.
#include "cs_common.cuh"

namespace cs {
namespace {

constexpr int FILL_THREADS = 256;

// words [0, n) of p set to v: the unaligned head and tail one word at a time, the body 16 bytes
// per store
__global__ void __launch_bounds__(FILL_THREADS) k_fill_u32(uint32_t *__restrict__ p, uint32_t v, size_t n) {
    const size_t head = min(n, (size_t)((16u - ((uintptr_t)p & 15u)) & 15u) / 4u);
    const size_t body = (n - head) / 4, tail = n - head - 4 * body;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    if (tid < head) p[tid] = v;
    uint4 *q = reinterpret_cast<uint4 *>(p + head);
    const uint4 v4 = make_uint4(v, v, v, v);
    for (size_t i = tid; i < body; i += stride) q[i] = v4;
    if (tid < tail) p[head + 4 * body + tid] = v;
}

constexpr int VIEWS_PER_LAUNCH = 16;  // 16 descriptors: well inside the 4 KB of kernel parameters
struct ViewBatch {
    ViewDesc v[VIEWS_PER_LAUNCH];
};
static_assert(sizeof(ViewBatch) <= 4000, "the descriptors of one launch fit the 4 KB of kernel parameters");

__global__ void k_put_views(ViewBatch b, int n, ViewDesc *__restrict__ dst) {
    constexpr int WORDS = sizeof(ViewDesc) / 4;
    static_assert(sizeof(ViewDesc) % 4 == 0, "descriptor of whole words");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(b.v);
    uint32_t *out = reinterpret_cast<uint32_t *>(dst);
    for (int i = threadIdx.x; i < n * WORDS; i += blockDim.x) out[i] = src[i];
}

__global__ void k_publish(const uint32_t *__restrict__ src, volatile uint32_t *dst, int words) {
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    __threadfence_system();
}

}  // namespace

cudaError_t fill_words(void *p, uint32_t v, size_t bytes, cudaStream_t s) {
    const size_t n = bytes / 4;
    if (n == 0) return cudaSuccess;
    const size_t blocks = min((n / 4 + FILL_THREADS - 1) / FILL_THREADS + 1, (size_t)4096);
    k_fill_u32<<<(unsigned)blocks, FILL_THREADS, 0, s>>>(static_cast<uint32_t *>(p), v, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t put_views(ViewDesc *dst, const ViewDesc *src, int n, cudaStream_t s) {
    for (int i = 0; i < n; i += VIEWS_PER_LAUNCH) {
        const int m = min(VIEWS_PER_LAUNCH, n - i);
        ViewBatch b;
        for (int j = 0; j < m; ++j) b.v[j] = src[i + j];
        k_put_views<<<1, 256, 0, s>>>(b, m, dst + i);
        count_launches(1);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t publish_words(const void *src, void *dst_host_mapped, int words, cudaStream_t s) {
    if (words <= 0) return cudaSuccess;
    k_publish<<<1, 32, 0, s>>>(static_cast<const uint32_t *>(src), static_cast<uint32_t *>(dst_host_mapped), words);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace cs
