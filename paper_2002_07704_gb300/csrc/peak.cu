// Measured arithmetic peaks of this GPU, for the roofline of the FMA kernels: a loop of
// independent fused multiply-adds in float32 or float64, timed with CUDA events.  No
// counterpart in the paper; a measurement utility beside the method's kernels.
#include <cuda_runtime.h>

#include "lsq_internal.h"

namespace lsq {
namespace {

constexpr int kChains = 8;     // independent accumulators per thread
constexpr int kIters = 4096;   // loop trips per launch

template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(T a, T b, T *__restrict__ sink) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (T)-1.2345) sink[0] = s;  // keeps the loop; never true for these inputs
}

}  // namespace
}  // namespace lsq

using namespace lsq;

extern "C" int lsq_measure_peak(int precision, double *tflops_host, void *stream) {
    clear_error();
    if (!tflops_host) return set_error(LSQ_ERR_INVALID_ARG, "tflops_host is null");
    if (precision != LSQ_F64 && precision != LSQ_F32)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64 or LSQ_F32");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    LSQ_CUDA_TRY(cudaGetDevice(&dev));
    LSQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevBuf<double> sink;
    LSQ_TRY(sink.alloc(1));
    const int blocks = sms * 8, threads = 256;
    cudaEvent_t e0, e1;
    LSQ_CUDA_TRY(cudaEventCreate(&e0));
    LSQ_CUDA_TRY(cudaEventCreate(&e1));
    auto launch = [&]() {
        note_launch();
        if (precision == LSQ_F64)
            k_fma_loop<double><<<blocks, threads, 0, s>>>(0.999999, 1e-7, sink.p);
        else
            k_fma_loop<float><<<blocks, threads, 0, s>>>(0.9999f, 1e-4f, reinterpret_cast<float *>(sink.p));
    };
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        LSQ_CUDA_TRY(cudaEventRecord(e0, s));
        launch();
        LSQ_CUDA_TRY(cudaEventRecord(e1, s));
        LSQ_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        LSQ_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best) best = ms;  // the first launch warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LSQ_CHECK_LAUNCH();
    const double fmas = (double)blocks * threads * kIters * kChains;
    *tflops_host = 2.0 * fmas / (best * 1e-3) / 1e12;
    return LSQ_OK;
}
