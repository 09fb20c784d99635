// FP64 throughput probe: the denominator of the plain path's roofline.
// Every thread runs eight independent FMA chains, so the FP64 pipe of every
// SM is saturated and nothing else limits the rate.
#include "common.cuh"

namespace spin {
namespace {

__global__ void dfma_probe_kernel(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    double x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; i++) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

}  // namespace
}  // namespace spin

extern "C" int spin_probe_fp64_peak(double* tflops, spin_stream_t stream) {
    using namespace spin;
    if (tflops == nullptr) return SPIN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    SPIN_CUDA_TRY(cudaGetDevice(&dev));
    SPIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 4, threads = 256, iters = 20000;
    double* out = nullptr;
    SPIN_CUDA_TRY(cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0, s);
        dfma_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            record_cuda_error(e, "dfma probe", __FILE__, __LINE__);
            cudaFree(out);
            return SPIN_ERR_CUDA;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    return SPIN_OK;
}
