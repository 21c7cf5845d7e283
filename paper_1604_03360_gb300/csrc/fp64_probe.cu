// fp64_probe.cu -- measures the FP64 FMA issue rate of this GPU (the
// roofline denominator of the FP64-bound stage kernel), and evaluates the
// kernels' hand-written reciprocal on given inputs so that tests can bound its
// error against IEEE division.  Neither is part of the method.  In the probe
// each thread runs 8 independent dependent-FMA chains; only one value per
// thread is written, to a buffer sized for the launch.
#include <cuda_runtime.h>

#include "../../include/hydro.h"
#include "hydro_math.cuh"

namespace {
__global__ void dfma_chains(double* out, int iters, double a, double b)
{
    double x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = threadIdx.x * 1e-9 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void rcp_eval(const double* __restrict__ x, double* __restrict__ y, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = hydro::rcp(x[i]);
}
}  // namespace

extern "C" hydro_status hydro_eval_rcp(const double* x, double* y, int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !y))) return HYDRO_ERR_INVALID_ARG;
    if (n == 0) return HYDRO_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HYDRO_ERR_CUDA;
    const long long want = (n + 255) / 256;
    const int blocks = (int)(want < 8LL * sms ? want : 8LL * sms);
    rcp_eval<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, y, n);
    return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ERR_CUDA;
}

extern "C" hydro_status hydro_measure_fp64_peak(void* stream, double* fma_per_second)
{
    if (!fma_per_second) return HYDRO_ERR_INVALID_ARG;
    *fma_per_second = 0.0;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HYDRO_ERR_CUDA;
    const int threads = 256, blocks = sms * 4, iters = 20000;
    double* buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * (size_t)threads * blocks) != cudaSuccess) return HYDRO_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dfma_chains<<<blocks, threads, 0, s>>>(buf, 200, 1.0000001, 1e-9);   // warm-up
    cudaEventRecord(e0, s);
    dfma_chains<<<blocks, threads, 0, s>>>(buf, iters, 1.0000001, 1e-9);
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (e != cudaSuccess || ms <= 0.f) return HYDRO_ERR_CUDA;
    *fma_per_second = (double)threads * blocks * iters * 8 / (ms * 1e-3);
    return HYDRO_OK;
}
