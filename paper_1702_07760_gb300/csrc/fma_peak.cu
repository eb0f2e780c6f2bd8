// FP32 fused multiply-add throughput of the current GPU: the denominator of
// the roofline of the force sweeps, which are bound by plain FP32 arithmetic
// and instruction issue rather than by HBM or the tensor cores.
//
// Every thread runs CHAINS independent dependency chains a <- a * b + c, so
// each warp scheduler always has independent FMAs to issue; the grid holds
// blocks_per_sm resident blocks of 256 threads on every SM.  Nothing is read
// from memory; one device word is written only if the chains reach a value
// they cannot reach (so the compiler keeps the arithmetic).
#include "sph.h"

#include <cuda_runtime.h>

#include <string>

namespace sphgb {
int set_error(int code, const std::string &msg);  // message for sph_last_error()
}

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int CHAINS = 16;

// Sink of the (never taken) store that keeps the chains live.
__device__ float g_peak_sink;

__global__ void __launch_bounds__(PEAK_THREADS) k_fma_chains(int iters, float b, float c, float never)
{
    float a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == never) g_peak_sink = s;
}

}  // namespace

extern "C" {

int sph_fp32_peak(int blocks_per_sm, int iters, void *stream, double *tflops, double *ms)
{
    if (!tflops || !ms) return sphgb::set_error(SPH_EINVAL, "tflops and ms must not be NULL");
    if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || iters > (1 << 20))
        return sphgb::set_error(SPH_EINVAL, "blocks_per_sm must be in [1, 8] and iters in [1, 2^20]");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return sphgb::set_error(SPH_ECUDA, cudaGetErrorString(e));
    const int blocks = sms * blocks_per_sm;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // the chains never reach a negative value (a, b, c >= 0), so the sink is not written
    if (e == cudaSuccess) {
        k_fma_chains<<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.999f, 1e-3f, -1.f);  // warm-up
        e = cudaEventRecord(e0, st);
    }
    if (e == cudaSuccess) {
        k_fma_chains<<<blocks, PEAK_THREADS, 0, st>>>(iters, 0.999f, 1e-3f, -1.f);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return sphgb::set_error(SPH_ECUDA, cudaGetErrorString(e));
    const double flops = 2.0 * CHAINS * (double)iters * PEAK_THREADS * blocks;
    *ms = t;
    *tflops = flops / (t * 1e-3) / 1e12;
    return SPH_OK;
}

}  // extern "C"
