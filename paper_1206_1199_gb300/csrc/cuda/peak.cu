// Arithmetic throughput probe: the measured counterpart of the peak that the
// FP32 force form's roofline divides by (152 SMs x 128 FP32 lanes x 2 flop
// per clock on GB300), and of the FP64 and reciprocal-square-root rates the
// design weighs against it.  Every thread runs kChains independent chains of
// dependent operations on a persistent grid of resident blocks: fused
// multiply-adds, scalar (fma.rn.f32, 2 flop) or packed (fma.rn.f32x2, 4
// flop), FP64 fused multiply-adds (fma.rn.f64, 2 flop), or hardware
// reciprocal square roots (rsqrt.approx.ftz.f32, 1 operation).  The caller
// times the launch with CUDA events on its stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "../common.h"

using namespace otoo;

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

typedef unsigned long long f2;

__device__ __forceinline__ f2 pack2(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float fold2(f2 v)
{
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo + hi;
}

// a <- a * b + c on every chain; b slightly below 1 and c small keep the
// values finite and normal for any iteration count.
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe_f32(int iters, float seed, float* sink)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed * (float)(tid + k + 1);
    const float b = 0.99999994f, c = 1.0e-7f;
    // unrolled so that the loop's own instructions take under 3% of issue
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[k]) : "f"(b), "f"(c));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0f) sink[tid] = s;  // never true: keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) k_fma_probe_f32x2(int iters, float seed, float* sink)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    f2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = pack2(seed * (float)(tid + k + 1), seed * (float)(tid + k + 2));
    const f2 b = pack2(0.99999994f, 0.99999994f), c = pack2(1.0e-7f, 1.0e-7f);
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[k]) : "l"(b), "l"(c));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += fold2(a[k]);
    if (s == -1.0f) sink[tid] = s;
}

// a <- a * b + c in FP64 on every chain
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe_f64(int iters, float seed, float* sink)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (double)seed * (double)(tid + k + 1);
    const double b = 0.9999999999999999, c = 1.0e-16;
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(a[k]) : "d"(b), "d"(c));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) sink[tid] = (float)s;
}

// a <- rsqrt(a) on every chain: the values tend to 1 and stay positive
__global__ void __launch_bounds__(kProbeThreads) k_rsqrt_probe(int iters, float seed, float* sink)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0f + seed * (float)(tid + k + 1);
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(a[k]));
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0f) sink[tid] = s;
}

typedef void (*ProbeKernel)(int, float, float*);

ProbeKernel probe_kernel(int kind)
{
    return kind == 0 ? k_fma_probe_f32 : kind == 1 ? k_fma_probe_f32x2 : kind == 2 ? k_fma_probe_f64 : k_rsqrt_probe;
}

int probe_grid(int kind, int* grid)
{
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return set_error(OTOO_ECUDA, "otoo_fma_probe: device query failed");
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_kernel(kind), kProbeThreads, 0);
    if (e != cudaSuccess || occ < 1) return set_error(OTOO_ECUDA, "otoo_fma_probe: occupancy query failed");
    *grid = nsm * occ;
    return OTOO_OK;
}

}  // namespace

extern "C" {

int64_t otoo_fma_probe_threads(void)
{
    int gmax = 0;
    for (int kind = 0; kind < 4; ++kind) {
        int g = 0;
        if (probe_grid(kind, &g)) return -1;
        if (g > gmax) gmax = g;
    }
    return (int64_t)gmax * kProbeThreads;
}

int otoo_fma_probe(int32_t iters, int32_t kind, float* sink, double* flops, void* stream)
{
    otoo::Range range_("otoo_fma_probe");
    OTOO_REQUIRE(iters >= 1 && kind >= 0 && kind <= 3 && sink && flops, OTOO_EINVAL, "otoo_fma_probe: bad argument");
    int grid = 0;
    const int rc = probe_grid(kind, &grid);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    probe_kernel(kind)<<<grid, kProbeThreads, 0, s>>>(iters, 1.0e-3f, sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OTOO_ECUDA, "otoo_fma_probe: %s", cudaGetErrorString(e));
    const double per_op = kind == 1 ? 4.0 : kind == 3 ? 1.0 : 2.0;
    *flops = (double)grid * kProbeThreads * kChains * (double)iters * per_op;
    return OTOO_OK;
}

}  // extern "C"
