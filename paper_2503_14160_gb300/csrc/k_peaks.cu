// Throughput microbenchmarks of the FP32 and FP64 FMA pipes, the denominators the
// evaluation and update kernels are compared with. Each thread runs eight independent
// FMA chains (enough to cover the pipe latency) for a fixed number of steps; the grid is
// eight CTAs of 256 threads per SM. Only one value per thread is stored, so the kernels
// are compute-only.
#include "cp_internal.cuh"

namespace cp {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int steps, T a, T b, T *out)
{
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (T)threadIdx.x * (T)1e-3 + (T)i;
    for (int it = 0; it < steps; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int time_probe(int steps, double *tflops)
{
    int dev = 0, sms = 0;
    CP_CUDA(cudaGetDevice(&dev));
    CP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = sms * 8;
    T *out = nullptr;
    CP_CUDA(cudaMalloc(&out, sizeof(T) * (size_t)threads * blocks));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, 0);
        k_fma_probe<T><<<blocks, threads>>>(steps, (T)0.999, (T)1e-3, out);
        count_launch();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;   // rep 0 warms up
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_fail(e, "FMA probe");
    *tflops = 2.0 * 8.0 * steps * (double)threads * blocks / (best * 1e-3) / 1e12;
    return CP_OK;
}

}  // namespace
}  // namespace cp

extern "C" int cp_alu_peaks(double *fp32_tflops, double *fp64_tflops)
{
    using namespace cp;
    if (!fp32_tflops || !fp64_tflops) return set_error("NULL argument"), CP_ERR_ARG;
    int rc = time_probe<float>(20000, fp32_tflops);
    if (rc != CP_OK) return rc;
    return time_probe<double>(500, fp64_tflops);
}
