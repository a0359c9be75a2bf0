// acac_peak_probe: the GPU's fused multiply-add rate in double or float, measured.
//
// The FP64 path of the solver is bound by the FP64 pipe rather than by HBM almost
// everywhere, so its kernels are judged against an arithmetic peak.  This probe
// measures that peak on the device at hand (and at its clocks of the moment): every
// thread of a full-occupancy grid runs eight independent multiply-add chains, so the
// pipe, not the latency of one chain, sets the rate.  No memory traffic beyond one
// store per thread at the end.
#include <cuda_runtime.h>

#include "acac.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) fma_probe_kernel(T* __restrict__ out, int iters, T a, T b,
                                                                   int lanes) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if ((threadIdx.x & 31) >= lanes) {   // lanes left idle: what a partly filled warp costs
        out[t] = (T)0;
        return;
    }
    T x[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (T)(t & 1023) * (T)1e-3 + (T)c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
    out[t] = s;
}

template <typename T>
int run_probe(int iters, int lanes, double* tflops, double* ms_out, cudaStream_t s) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ACAC_E_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ACAC_E_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<T>, PROBE_THREADS, 0) != cudaSuccess)
        return ACAC_E_CUDA;
    if (per_sm < 1) per_sm = 1;
    const int blocks = sms * per_sm;
    const size_t threads = (size_t)blocks * PROBE_THREADS;
    T* out = nullptr;
    if (cudaMalloc(&out, threads * sizeof(T)) != cudaSuccess) return ACAC_E_NOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = ACAC_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = ACAC_E_CUDA;
    const T a = (T)0.999999, b = (T)1e-7;
    float ms = 0.f;
    if (st == ACAC_OK) {
        fma_probe_kernel<T><<<blocks, PROBE_THREADS, 0, s>>>(out, iters, a, b, lanes);   // warm-up
        cudaEventRecord(e0, s);
        fma_probe_kernel<T><<<blocks, PROBE_THREADS, 0, s>>>(out, iters, a, b, lanes);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            st = ACAC_E_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (st != ACAC_OK) return st;
    const double flops = 2.0 * PROBE_CHAINS * (double)iters * (double)threads * lanes / 32.0;
    if (tflops) *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    if (ms_out) *ms_out = ms;
    return ACAC_OK;
}

}  // namespace

extern "C" int acac_peak_probe(int kind, int iters, double* tflops, double* ms, void* cuda_stream) {
    if (iters < 1) return ACAC_E_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (kind == 0) return run_probe<double>(iters, 32, tflops, ms, s);
    if (kind == 1) return run_probe<float>(iters, 32, tflops, ms, s);
    if (kind >= 2 && kind <= 6) return run_probe<double>(iters, 32 >> (kind - 1), tflops, ms, s);
    return ACAC_E_ARG;
}
