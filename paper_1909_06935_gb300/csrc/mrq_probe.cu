// mrq_probe.cu - measured ceilings of the device for the walk's roofline (include/mrq.h).
//
// The walk is FP64 arithmetic on gathered table entries, so two ceilings bound it: the FP64 FMA
// rate of the SMs and the rate of random 8-byte reads from tables that stay in L2 (the 56-orbital
// workload) or live in HBM (the 104-orbital one).  This file measures both on the device it runs
// on, with kernels shaped like the bound they probe: independent FMA chains in registers on every
// SM, and independent random reads (8 in flight per thread) from a table of a chosen size.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/mrq.h"

namespace {

// 8 independent FMA chains per thread; x -> a x + b keeps every chain bounded
__global__ void __launch_bounds__(256) k_probe_fma(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    if (s == -1.0) out[blockIdx.x & 1023u] = s;      // never true; keeps the chains alive
}

__device__ __forceinline__ unsigned long long probe_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// random 8-byte reads: each thread issues 8 independent reads per iteration
__global__ void __launch_bounds__(256) k_probe_gather(const double* __restrict__ tab, unsigned long long mask, int iters,
                                                     double* out) {
    const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    for (int i = 0; i < iters; i++) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = __ldg(tab + (probe_mix(t * 0x9E3779B97F4A7C15ull + (unsigned)(8 * i + k)) & mask));
#pragma unroll
        for (int k = 0; k < 8; k++) acc += v[k];
    }
    if (acc == -1.0) out[t & 1023] = acc;
}

__global__ void k_probe_fill(double* tab, unsigned long long n) {
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        tab[i] = 1e-9 * (double)(i & 1023);
}

}  // namespace

extern "C" int mrq_probe_peaks(int device, double* out3) {
    if (!out3) return MRQ_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return MRQ_CUDA_ERROR;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
        return MRQ_CUDA_ERROR;
    const unsigned long long l2_doubles = 1ull << 21;          // 16 MiB: resident in L2
    const unsigned long long hbm_doubles = 1ull << 29;         // 4 GiB: far larger than L2
    double *tab = nullptr, *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    auto timed = [&](auto launch, int reps) -> double {      // best of reps, seconds
        double best = 1e30;
        for (int r = 0; r < reps; r++) {
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, 1e-3 * ms);
        }
        return best;
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, 1024 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&tab, hbm_doubles * sizeof(double)) != cudaSuccess) {
        rc = MRQ_CUDA_ERROR;
    } else {
        k_probe_fill<<<4 * sms, 256, 0, st>>>(tab, hbm_doubles);
        // FP64 FMA: 8 blocks of 256 threads per SM, 8 chains each
        const int fma_iters = 4096;
        const unsigned fblocks = 8u * (unsigned)sms;
        k_probe_fma<<<fblocks, 256, 0, st>>>(sink, 64, 0.999999, 1e-7);        // warm-up
        const double tf = timed([&] { k_probe_fma<<<fblocks, 256, 0, st>>>(sink, fma_iters, 0.999999, 1e-7); }, 3);
        out3[0] = 2.0 * 8.0 * fma_iters * (double)fblocks * 256.0 / tf;
        // random 8-byte reads from an L2-resident and an HBM-resident table
        const int l2_iters = 256, hbm_iters = 64;
        const unsigned gblocks = 16u * (unsigned)sms;
        const double per_iter = 8.0 * (double)gblocks * 256.0;
        k_probe_gather<<<gblocks, 256, 0, st>>>(tab, l2_doubles - 1, 4, sink);
        const double tl = timed([&] { k_probe_gather<<<gblocks, 256, 0, st>>>(tab, l2_doubles - 1, l2_iters, sink); }, 3);
        const double th = timed([&] { k_probe_gather<<<gblocks, 256, 0, st>>>(tab, hbm_doubles - 1, hbm_iters, sink); }, 3);
        out3[1] = per_iter * l2_iters / tl;
        out3[2] = per_iter * hbm_iters / th;
        if (cudaGetLastError() != cudaSuccess) rc = MRQ_CUDA_ERROR;
    }
    if (tab) cudaFree(tab);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return rc;
}
