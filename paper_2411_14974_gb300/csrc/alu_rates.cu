// Measured per-SM issue rates of the two arithmetic pipes the blend kernels load: the
// transcendental unit (ex2.approx, the exponentials of the LogSumExp and the sigmoid, Eq. S1/S2)
// and the FP32 fused multiply-add pipe.  The rates are the roofline denominators of those
// kernels, so they are measured here rather than taken from a table.
//
// Each thread runs 8 independent dependency chains (enough in flight to fill the pipe) for a fixed
// number of steps: x = 2^-x for the transcendental unit (bounded in [0.5, 1]), x = a x + b for the
// FMA pipe.  Every block records the SM it ran on and its first and last clock64(); per SM the
// results executed divided by the cycles between its earliest start and latest end give the rate
// per clock.  The wall time of the launch (CUDA events) divided into those cycles gives the SM
// clock during the run.
#include <algorithm>
#include <vector>

#include "cs_api_internal.h"
#include "cs_common.cuh"

using namespace cs;

namespace {

constexpr int RATE_THREADS = 256;
constexpr int RATE_CHAINS = 8;
constexpr int RATE_STEPS = 2048;

struct BlockClock {
    long long start, end;
    unsigned smid;
};

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

template <bool MUFU>
__global__ void __launch_bounds__(RATE_THREADS) k_alu_rate(float seed, float *sink, BlockClock *clocks) {
    float x[RATE_CHAINS];
#pragma unroll
    for (int c = 0; c < RATE_CHAINS; ++c) x[c] = seed + 0.01f * c + 1e-6f * threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < RATE_STEPS; ++i) {
#pragma unroll
        for (int c = 0; c < RATE_CHAINS; ++c) {
            if (MUFU) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(-x[c]));
            else x[c] = fmaf(x[c], 0.999f, 0.001f);
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < RATE_CHAINS; ++c) s += x[c];
    if (s == -1.0f) sink[threadIdx.x] = s;  // never true: keeps the chains live
    if (threadIdx.x == 0) clocks[blockIdx.x] = BlockClock{t0, t1, smid()};
}

// median over SMs of (results per SM) / (cycles the SM spent), and the cycles of the slowest SM
template <bool MUFU>
cudaError_t measure(int blocks, float *sink, BlockClock *dclk, cudaStream_t s, double *rate, double *clock_mhz) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_alu_rate<MUFU><<<blocks, RATE_THREADS, 0, s>>>(0.5f, sink, dclk);  // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        k_alu_rate<MUFU><<<blocks, RATE_THREADS, 0, s>>>(0.5f, sink, dclk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    std::vector<BlockClock> h(blocks);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dclk, sizeof(BlockClock) * blocks, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    count_launches(2);
    struct Sm {
        long long lo = 0, hi = 0;
        int n = 0;
    };
    std::vector<Sm> sms;
    for (const BlockClock &b : h) {
        if (b.smid >= sms.size()) sms.resize(b.smid + 1);
        Sm &m = sms[b.smid];
        m.lo = m.n ? std::min(m.lo, b.start) : b.start;
        m.hi = m.n ? std::max(m.hi, b.end) : b.end;
        m.n++;
    }
    std::vector<double> rates;
    long long span = 0;
    for (const Sm &m : sms) {
        if (!m.n || m.hi <= m.lo) continue;
        const double results = (double)m.n * RATE_THREADS * RATE_CHAINS * RATE_STEPS;
        rates.push_back(results / (double)(m.hi - m.lo));
        span = std::max(span, m.hi - m.lo);
    }
    if (rates.empty()) return cudaErrorUnknown;
    std::sort(rates.begin(), rates.end());
    *rate = rates[rates.size() / 2];
    *clock_mhz = ms > 0.f ? (double)span / (ms * 1e3) : 0.0;
    return cudaSuccess;
}

}  // namespace

extern "C" cs_status cs_measure_alu_rates(int32_t device, double *out) {
    if (!out) return fail(CS_ERR_ARG, "out is NULL");
    DeviceGuard dg(device);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return fail_cuda(e, "cudaDeviceGetAttribute");
    const int blocks = sms * 8;  // 8 blocks of 256 threads per SM: 64 warps, the pipes stay fed
    float *sink = nullptr;
    BlockClock *dclk = nullptr;
    cudaStream_t s = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&sink, RATE_THREADS * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dclk, sizeof(BlockClock) * blocks);
    double mufu = 0, mufu_mhz = 0, fma = 0, fma_mhz = 0;
    if (e == cudaSuccess) e = measure<true>(blocks, sink, dclk, s, &mufu, &mufu_mhz);
    if (e == cudaSuccess) e = measure<false>(blocks, sink, dclk, s, &fma, &fma_mhz);
    if (sink) cudaFree(sink);
    if (dclk) cudaFree(dclk);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return fail_cuda(e, "cs_measure_alu_rates");
    out[0] = mufu;
    out[1] = fma;
    out[2] = 0.5 * (mufu_mhz + fma_mhz);
    out[3] = (double)sms;
    return CS_OK;
}
