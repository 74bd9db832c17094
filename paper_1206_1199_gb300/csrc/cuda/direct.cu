// Direct summation on the device: chosen targets against every particle of
// a system, in FP64 -- the exact reference the learned opening angle is
// trained against (the measured group errors are this sum's, the paper's
// O(N^2) brute force of Section II), and a check of the tree force.
//
// Kernels
//   k_direct_part  block (target tile of 128, source chunk): the chunk's
//                  sources staged through shared memory, FP64 pairs, one
//                  partial sum per (chunk, target).
//   k_direct_sum   the chunk partials of each target summed in chunk order.
#include <cuda_runtime.h>

#include <cstdint>

#include "../common.h"

using namespace otoo;

namespace {

constexpr int kTgt = 128;     // targets per block
constexpr int kTile = 128;    // sources staged per tile

__global__ void __launch_bounds__(kTgt) k_direct_part(const otoo_src* __restrict__ src, int64_t n_src,
                                                      const int64_t* __restrict__ tgt, int64_t n_tgt, double eps2,
                                                      int64_t chunk, double* __restrict__ part,
                                                      uint32_t* __restrict__ status)
{
    __shared__ double4 s[kTile];
    const int64_t t = (int64_t)blockIdx.x * kTgt + threadIdx.x;
    const int64_t j0 = (int64_t)blockIdx.y * chunk;
    const int64_t j1 = j0 + chunk < n_src ? j0 + chunk : n_src;
    int64_t ti = -1;
    double xi = 0, yi = 0, zi = 0;
    if (t < n_tgt) {
        ti = tgt[t];
        if (ti < 0 || ti >= n_src) {
            atomicOr(status, 2u);
            ti = -1;
        } else {
            xi = src[ti].x;
            yi = src[ti].y;
            zi = src[ti].z;
        }
    }
    double ax = 0, ay = 0, az = 0, ph = 0;
    for (int64_t b = j0; b < j1; b += kTile) {
        const int64_t j = b + threadIdx.x;
        if (j < j1) {
            const otoo_src q = src[j];
            s[threadIdx.x] = make_double4(q.x, q.y, q.z, (double)q.m);
        }
        __syncthreads();
        const int cnt = j1 - b < kTile ? (int)(j1 - b) : kTile;
        const int kself = (ti >= b && ti < b + cnt) ? (int)(ti - b) : -1;  // j != i
        for (int k = 0; k < cnt; ++k) {
            const double4 q = s[k];
            const double rx = q.x - xi, ry = q.y - yi, rz = q.z - zi;
            const double r2 = rx * rx + ry * ry + rz * rz + eps2;
            const double inv = rsqrt(r2);
            const double mi = (k == kself ? 0.0 : q.w) * inv;
            const double mi3 = mi * inv * inv;
            ax += mi3 * rx;
            ay += mi3 * ry;
            az += mi3 * rz;
            ph -= mi;
        }
        __syncthreads();
    }
    if (t < n_tgt) {
        double* d = part + ((int64_t)blockIdx.y * n_tgt + t) * 4;
        d[0] = ax;
        d[1] = ay;
        d[2] = az;
        d[3] = ph;
    }
}

__global__ void k_direct_sum(const double* __restrict__ part, int64_t n_tgt, int n_chunk, double* __restrict__ accel,
                             double* __restrict__ pot)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tgt) return;
    double a[4] = {0, 0, 0, 0};
    for (int c = 0; c < n_chunk; ++c)
        for (int k = 0; k < 4; ++k) a[k] += part[((int64_t)c * n_tgt + t) * 4 + k];
    accel[3 * t] = a[0];
    accel[3 * t + 1] = a[1];
    accel[3 * t + 2] = a[2];
    pot[t] = a[3];
}

#define CUDA_TRY(expr)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return set_error(OTOO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

}  // namespace

extern "C" {

int64_t otoo_direct_chunks(int64_t n_src, int64_t n_tgt)
{
    if (n_src < 1 || n_tgt < 1) return 0;
    // enough blocks to fill the GPU several times over
    const int64_t tblocks = (n_tgt + kTgt - 1) / kTgt;
    int64_t chunks = (4 * 152 + tblocks - 1) / tblocks;
    if (chunks < 1) chunks = 1;
    const int64_t maxc = (n_src + kTile - 1) / kTile;
    return chunks < maxc ? chunks : maxc;
}

int otoo_direct(const otoo_src* src, int64_t n_src, const int64_t* targets, int64_t n_tgt, double eps2, double* accel,
                double* pot, double* scratch, uint32_t* status, void* stream)
{
    otoo::Range range_("otoo_direct");
    OTOO_REQUIRE(src && targets && accel && pot && scratch && status, OTOO_EINVAL, "otoo_direct: NULL pointer");
    OTOO_REQUIRE(n_src >= 1 && n_tgt >= 1 && n_tgt <= ((int64_t)1 << 31), OTOO_EINVAL, "otoo_direct: bad sizes");
    OTOO_REQUIRE(eps2 > 0.0, OTOO_EINVAL, "otoo_direct: eps2 must be > 0");
    const int64_t nc = otoo_direct_chunks(n_src, n_tgt);
    const int64_t chunk = ((n_src + nc - 1) / nc + kTile - 1) / kTile * kTile;
    const int64_t nch = (n_src + chunk - 1) / chunk;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
    dim3 grid((unsigned)((n_tgt + kTgt - 1) / kTgt), (unsigned)nch);
    k_direct_part<<<grid, kTgt, 0, s>>>(src, n_src, targets, n_tgt, eps2, chunk, scratch, status);
    CUDA_TRY(cudaGetLastError());
    k_direct_sum<<<(unsigned)((n_tgt + 127) / 128), 128, 0, s>>>(scratch, n_tgt, (int)nch, accel, pot);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

}  // extern "C"
