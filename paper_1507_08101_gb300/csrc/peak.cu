// Measured float64 rate of the device (no counterpart in the paper): the
// float64 products of this library are bound by the float64 pipe on GB300, so
// their roofline needs the pipe's rate on the machine at hand rather than a
// nominal figure.
//
// k_dfma_chains: every thread runs kChains (16) independent chains of fused
// multiply-adds a <- a * b + c (kChains in flight hide the pipe latency), for
// `iters` steps; the grid holds every SM with 2048 threads.  b slightly below 1
// and c small keep the values bounded and normal.  One thread whose result can
// never match writes it, so the compiler cannot drop the work.
#include "common.cuh"

namespace sp {

constexpr int kChains = 16;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_dfma_chains(int iters, double b, double c, double *sink) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    // four steps per loop trip, so the loop's own integer work is a small
    // share of the issue slots
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __fma_rn(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) *sink = s;  // never true: the values stay near 1
}

}  // namespace sp

extern "C" int sp_device_fp64_rate(double *tflops, double *ms, void *stream) {
    if (!tflops) return SP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 1;
    SP_TRY(sp::device_sm_count(&sms));
    const int blocks = sms * (2048 / sp::kPeakThreads);
    const int iters = 1 << 13;
    sp::Tmp sink(s);
    SP_TRY(sink.alloc(sizeof(double)));
    cudaEvent_t e0, e1;
    SP_CUDA(cudaEventCreate(&e0));
    SP_CUDA(cudaEventCreate(&e1));
    float best = 0.0f;
    int rc = SP_OK;
    for (int rep = 0; rep < 4 && rc == SP_OK; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, s);
        sp::k_dfma_chains<<<blocks, sp::kPeakThreads, 0, s>>>(iters, 0.9999999, 1e-7, sink.as<double>());
        cudaEventRecord(e1, s);
        cudaError_t err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaGetLastError();
        if (err != cudaSuccess) {
            sp_internal_note_cuda_error(err, "k_dfma_chains", __FILE__, __LINE__);
            rc = SP_ERR_CUDA;
            break;
        }
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && (best == 0.0f || t < best)) best = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SP_OK) return rc;
    const double flops = 2.0 * sp::kChains * (double)iters * blocks * sp::kPeakThreads;
    *tflops = flops / (best * 1e-3) / 1e12;
    if (ms) *ms = best;
    return SP_OK;
}
