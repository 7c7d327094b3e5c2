// FP64 fused multiply-add throughput of the current GPU: the peak that bounds
// the FP64 path's contraction (no FP64 figure is measured elsewhere).  Each
// thread runs eight independent FMA chains in registers, so the FP64 pipes, not
// latency or memory, limit the loop.
#include "kernels.cuh"

namespace afq {

__global__ void __launch_bounds__(256) dfma_loop_kernel(int iters, double a, double b, double* out) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 1e-3 * (threadIdx.x + 1) + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == -1.0) out[blockIdx.x] = s;   // never true: keeps the chains alive
}

}  // namespace afq

using namespace afq;

extern "C" afqmc_status afqmc_fp64_fma_rate(double* tflops, void* stream) {
    if (!tflops) return set_error(AFQMC_ERR_ARG, "tflops is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return set_error(AFQMC_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = 1 << 15, blocks = sms * 8, threads = 256;
    double best = 0.0;
    for (int rep = 0; rep < 4; ++rep) {   // the first launch warms up
        cudaEventRecord(e0, s);
        dfma_loop_kernel<<<blocks, threads, 0, s>>>(iters, 1.0 - 0x1p-40, 0x1p-40, nullptr);
        count_launches(1);
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flop = 2.0 * 8.0 * iters * (double)blocks * threads;
        if (rep > 0 && ms > 0.f) best = fmax(best, flop / (ms * 1e-3) / 1e12);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess)
        return set_error(AFQMC_ERR_CUDA, "FMA loop: %s", cudaGetErrorString(e));
    *tflops = best;
    return AFQMC_OK;
}
