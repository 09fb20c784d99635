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

// The same on the FP64 tensor path (DMMA): every warp issues eight
// independent mma.sync m8n8k4 f64 chains (256 FMAs per instruction).  On
// GB300 DMMA and DFMA share one FP64 unit, and this rate is the lower one,
// which is why the level products are DFMA kernels.
__global__ void dmma_probe_kernel(double* out, int iters, double a, double b) {
    double c[8][2];
#pragma unroll
    for (int j = 0; j < 8; j++) c[j][0] = c[j][1] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int j = 0; j < 8; j++)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(a), "d"(b));
    }
    double acc = 0.0;
#pragma unroll
    for (int j = 0; j < 8; j++) acc += c[j][0] + c[j][1];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// Best of three timed launches (after one warm-up) of `launch` on every SM;
// returns TFLOP/s for `flops` per launch.
template <class F>
int time_probe(F launch, double flops, cudaStream_t s, double* tflops) {
    cudaEvent_t e0, e1;
    SPIN_CUDA_TRY(cudaEventCreate(&e0));
    SPIN_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int rc = SPIN_OK;
    for (int rep = 0; rep < 4 && rc == SPIN_OK; rep++) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) {
            record_cuda_error(e, "fp64 probe", __FILE__, __LINE__);
            rc = SPIN_ERR_CUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == SPIN_OK) *tflops = flops / (best * 1e-3) / 1e12;
    return rc;
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
    const int rc = time_probe([&] { dfma_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.9999999, 1e-7); },
                              2.0 * 8.0 * iters * (double)blocks * threads, s, tflops);
    cudaFree(out);
    return rc;
}

extern "C" int spin_probe_fp64_mma_peak(double* tflops, spin_stream_t stream) {
    using namespace spin;
    if (tflops == nullptr) return SPIN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    SPIN_CUDA_TRY(cudaGetDevice(&dev));
    SPIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 4, threads = 256, iters = 2500;  // the DFMA probe's flops
    double* out = nullptr;
    SPIN_CUDA_TRY(cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)));
    // per warp and chain step: one m8n8k4 = 8 * 8 * 4 FMAs
    const double warps = (double)blocks * threads / 32.0;
    const int rc = time_probe([&] { dmma_probe_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.5, 0.25); },
                              2.0 * 256.0 * 8.0 * iters * warps, s, tflops);
    cudaFree(out);
    return rc;
}
