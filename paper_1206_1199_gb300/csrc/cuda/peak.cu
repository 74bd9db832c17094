// FP32 FMA throughput probe: the measured counterpart of the peak that the
// FP32 force form's roofline divides by (152 SMs x 128 FP32 lanes x 2 flop
// per clock on GB300).  Every thread runs kChains independent chains of
// dependent fused multiply-adds, scalar (fma.rn.f32, 2 flop) or packed
// (fma.rn.f32x2, 4 flop), on a persistent grid of resident blocks.  The
// caller times the launch with CUDA events on its stream.
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

int probe_grid(int packed, int* grid)
{
    int dev = 0, nsm = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return set_error(OTOO_ECUDA, "otoo_fma_probe: device query failed");
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, packed ? k_fma_probe_f32x2 : k_fma_probe_f32, kProbeThreads, 0);
    if (e != cudaSuccess || occ < 1) return set_error(OTOO_ECUDA, "otoo_fma_probe: occupancy query failed");
    *grid = nsm * occ;
    return OTOO_OK;
}

}  // namespace

extern "C" {

int64_t otoo_fma_probe_threads(void)
{
    int g0 = 0, g1 = 0;
    if (probe_grid(0, &g0) || probe_grid(1, &g1)) return -1;
    return (int64_t)(g0 > g1 ? g0 : g1) * kProbeThreads;
}

int otoo_fma_probe(int32_t iters, int32_t packed, float* sink, double* flops, void* stream)
{
    otoo::Range range_("otoo_fma_probe");
    OTOO_REQUIRE(iters >= 1 && (packed == 0 || packed == 1) && sink && flops, OTOO_EINVAL,
                 "otoo_fma_probe: bad argument");
    int grid = 0;
    const int rc = probe_grid(packed, &grid);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (packed)
        k_fma_probe_f32x2<<<grid, kProbeThreads, 0, s>>>(iters, 1.0e-3f, sink);
    else
        k_fma_probe_f32<<<grid, kProbeThreads, 0, s>>>(iters, 1.0e-3f, sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(OTOO_ECUDA, "otoo_fma_probe: %s", cudaGetErrorString(e));
    *flops = (double)grid * kProbeThreads * kChains * (double)iters * (packed ? 4.0 : 2.0);
    return OTOO_OK;
}

}  // extern "C"
