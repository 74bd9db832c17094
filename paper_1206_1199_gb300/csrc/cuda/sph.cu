// SPH density on the device (Section II, "Bounding Radius for SPH"):
// rho_i = sum_j m_j W(|x_i - x_j|, h_j) (Eq. SPH_SUM with A = m) over the
// particle lists of the SPH walk (Eq. SPH_RAD), which hold every source j
// whose support can reach a particle of the group.  Readings: the M4 cubic
// spline with support radius h, the scatter form (each source's own h_j), the
// source itself included.
//
// Kernels
//   k_h_tree          h in tree order (through the permutation).
//   k_density<IB>     one work item (group, target chunk, list chunk) per warp
//                     from an atomic ticket; 32-entry tiles staged in shared
//                     memory as (x_j - c, m_j 8/(pi h_j^3), 1/h_j) in FP32
//                     relative to the group centre c, keeping only entries
//                     within (1 + 2^-10) h_j of the item's own target box (the
//                     others have W = 0 at every target; the walk's lists are
//                     cut at cell level and hold about 12 times more entries
//                     than neighbours); each lane sums IB targets, FP32
//                     within a tile, FP64 across tiles.
//   k_density_merge   FP64 sum of the list chunks of split groups, in chunk
//                     order.
//   k_sph_direct      FP64 brute force over all sources for chosen targets
//                     (the reference of the checks): one thread per target,
//                     sources staged through shared memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "../common.h"

using namespace otoo;

namespace {

constexpr int kDW = 4;  // warps per CTA
constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kBadItem = 1u;   // same status bits as the force step
constexpr uint32_t kBadIndex = 2u;
constexpr float kNorm = 2.546479089470325f;  // 8 / pi

__global__ void k_h_tree(const float* __restrict__ h, const int64_t* __restrict__ perm, int64_t n,
                         float* __restrict__ ht, uint32_t* __restrict__ status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm ? perm[k] : k;
    if (i < 0 || i >= n) {
        atomicOr(status, kBadIndex);
        ht[k] = 1.0f;
        return;
    }
    ht[k] = h[i];
}

// M4 cubic spline shape w(q), q = r / h (zero for q >= 1).
__device__ __forceinline__ float w_m4(float q)
{
    const float a = 1.0f - q;
    const float inner = fmaf(q * q, fmaf(6.0f, q, -6.0f), 1.0f);
    return q <= 0.5f ? inner : (q < 1.0f ? 2.0f * a * a * a : 0.0f);
}

template <int IB>
__global__ void __launch_bounds__(kDW * 32) k_density(otoo_dev_system sys, const float* __restrict__ ht,
                                                      double* __restrict__ rho)
{
    __shared__ float4 tp[kDW][32];
    __shared__ float tih[kDW][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* counter = sys.counter;
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(counter, 1u);
        t = __shfl_sync(kFull, t, 0);
        if (t >= sys.n_items) break;
        const otoo_item it = sys.items[t];
        bool ok = it.g >= 0 && it.g < sys.n_groups;
        otoo_group g{};
        if (ok) {
            g = sys.groups[it.g];
            const int64_t len = (int64_t)g.n_cell + g.n_part;
            ok = it.i0 >= 0 && it.ni >= 1 && it.ni <= 32 * IB && it.i0 + it.ni <= g.count && it.j0 >= 0 &&
                 it.j0 <= it.j1 && it.j1 <= len && g.list_off >= 0 && g.list_off + len <= sys.n_list &&
                 g.first >= 0 && (int64_t)g.first + g.count <= sys.n_part &&
                 (it.slot < 0 || g.count <= sys.n_crit_max);
        }
        if (!ok) {
            if (lane == 0) atomicOr(counter + 1, kBadItem);
            continue;
        }
        float xi[IB], yi[IB], zi[IB];
        double acc[IB];
        float blo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, bhi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
        for (int r = 0; r < IB; ++r) {
            const int k = lane + 32 * r;
            acc[r] = 0.0;
            xi[r] = yi[r] = zi[r] = 0.f;
            if (k < it.ni) {
                const otoo_src s = sys.src[g.first + it.i0 + k];
                xi[r] = (float)(s.x - g.cx);
                yi[r] = (float)(s.y - g.cy);
                zi[r] = (float)(s.z - g.cz);
                blo[0] = fminf(blo[0], xi[r]), bhi[0] = fmaxf(bhi[0], xi[r]);
                blo[1] = fminf(blo[1], yi[r]), bhi[1] = fmaxf(bhi[1], yi[r]);
                blo[2] = fminf(blo[2], zi[r]), bhi[2] = fmaxf(bhi[2], zi[r]);
            }
        }
        // the box of this item's targets (the same FP32 values the pairs use)
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                blo[a] = fminf(blo[a], __shfl_xor_sync(kFull, blo[a], o));
                bhi[a] = fmaxf(bhi[a], __shfl_xor_sync(kFull, bhi[a], o));
            }
        for (int32_t j = it.j0; j < it.j1; j += 32) {
            const int32_t jj = j + lane;
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            float ih = 0.f;
            bool keep = false;
            if (jj < it.j1) {
                const int32_t e = sys.list[g.list_off + jj];
                if (e >= 0 && e < sys.n_part) {
                    const otoo_src s = sys.src[e];
                    const float h = ht[e];
                    ih = 1.0f / h;
                    p = make_float4((float)(s.x - g.cx), (float)(s.y - g.cy), (float)(s.z - g.cz),
                                    s.m * kNorm * ih * ih * ih);
                    // distance from the entry to the target box against its support
                    const float dx = fmaxf(0.f, fmaxf(blo[0] - p.x, p.x - bhi[0]));
                    const float dy = fmaxf(0.f, fmaxf(blo[1] - p.y, p.y - bhi[1]));
                    const float dz = fmaxf(0.f, fmaxf(blo[2] - p.z, p.z - bhi[2]));
                    const float hm = h * (1.0f + 0x1p-10f);
                    keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < hm * hm;
                } else {
                    atomicOr(counter + 1, kBadIndex);
                }
            }
            const unsigned km = __ballot_sync(kFull, keep);
            if (keep) {
                const int slot = __popc(km & ((1u << lane) - 1u));
                tp[w][slot] = p;
                tih[w][slot] = ih;
            }
            __syncwarp();
            const int cnt = __popc(km);
            float part[IB];
#pragma unroll
            for (int r = 0; r < IB; ++r) part[r] = 0.f;
            for (int q = 0; q < cnt; ++q) {
                const float4 pj = tp[w][q];
                const float ihj = tih[w][q];
#pragma unroll
                for (int r = 0; r < IB; ++r) {
                    const float dx = pj.x - xi[r], dy = pj.y - yi[r], dz = pj.z - zi[r];
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float qq = r2 > 0.f ? r2 * rsqrtf(r2) * ihj : 0.f;
                    part[r] = fmaf(pj.w, w_m4(qq), part[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < IB; ++r) acc[r] += (double)part[r];
            __syncwarp();
        }
#pragma unroll
        for (int r = 0; r < IB; ++r) {
            const int k = lane + 32 * r;
            if (k >= it.ni) continue;
            const int64_t ti = (int64_t)g.first + it.i0 + k;
            if (it.slot < 0) {
                rho[sys.perm ? sys.perm[ti] : ti] = acc[r];
            } else {
                sys.partial[((int64_t)it.slot * sys.n_crit_max + it.i0 + k) * 4] = acc[r];
            }
        }
    }
}

__global__ void k_density_merge(otoo_dev_system sys, double* __restrict__ rho)
{
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= sys.n_splits) return;
    const otoo_split sp = sys.splits[wid];
    if (sp.g < 0 || sp.g >= sys.n_groups || sp.slot0 < 0 || sp.n_chunks < 1) {
        if (lane == 0) atomicOr(sys.counter + 1, kBadItem);
        return;
    }
    const otoo_group g = sys.groups[sp.g];
    if (g.count > sys.n_crit_max) {
        if (lane == 0) atomicOr(sys.counter + 1, kBadItem);
        return;
    }
    for (int i = lane; i < g.count; i += 32) {
        double s = 0.0;
        for (int c = 0; c < sp.n_chunks; ++c) s += sys.partial[((int64_t)(sp.slot0 + c) * sys.n_crit_max + i) * 4];
        const int64_t ti = (int64_t)g.first + i;
        rho[sys.perm ? sys.perm[ti] : ti] = s;
    }
}

// FP64 kernel value (same spline as the pairs above, in FP64).
__device__ __forceinline__ double w_m4_64(double r, double h)
{
    const double q = r / h;
    const double a = 1.0 - q;
    const double w = q <= 0.5 ? 1.0 - 6.0 * q * q + 6.0 * q * q * q : (q < 1.0 ? 2.0 * a * a * a : 0.0);
    return 8.0 / (3.141592653589793 * h * h * h) * w;
}

__global__ void __launch_bounds__(128) k_sph_direct(const otoo_src* __restrict__ src, const float* __restrict__ h,
                                                    int64_t n, const int64_t* __restrict__ tgt, int64_t n_tgt,
                                                    double* __restrict__ rho, uint32_t* __restrict__ status)
{
    __shared__ double4 s[128];
    __shared__ double sh[128];
    const int64_t t = (int64_t)blockIdx.x * 128 + threadIdx.x;
    int64_t i = -1;
    double xi = 0, yi = 0, zi = 0;
    if (t < n_tgt) {
        i = tgt[t];
        if (i < 0 || i >= n) {
            atomicOr(status, kBadIndex);
            i = -1;
        } else {
            xi = src[i].x, yi = src[i].y, zi = src[i].z;
        }
    }
    double sum = 0.0;
    for (int64_t b = 0; b < n; b += 128) {
        const int64_t j = b + threadIdx.x;
        if (j < n) {
            const otoo_src q = src[j];
            s[threadIdx.x] = make_double4(q.x, q.y, q.z, (double)q.m);
            sh[threadIdx.x] = (double)h[j];
        }
        __syncthreads();
        const int cnt = n - b < 128 ? (int)(n - b) : 128;
        for (int k = 0; k < cnt; ++k) {
            const double4 q = s[k];
            const double dx = q.x - xi, dy = q.y - yi, dz = q.z - zi;
            const double r = sqrt(dx * dx + dy * dy + dz * dz);
            if (r < sh[k]) sum += q.w * w_m4_64(r, sh[k]);
        }
        __syncthreads();
    }
    if (t < n_tgt) rho[t] = sum;
}

#define CUDA_TRY(expr)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return set_error(OTOO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

template <int IB>
int launch(const otoo_dev_system* sys, const float* ht, double* rho, cudaStream_t s)
{
    int dev = 0, sms = 0, occ = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_density<IB>, kDW * 32, 0));
    if (occ < 1) occ = 1;
    int64_t blocks = (int64_t)sms * occ;
    const int64_t need = ((int64_t)sys->n_items + kDW - 1) / kDW;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    k_density<IB><<<(unsigned)blocks, kDW * 32, 0, s>>>(*sys, ht, rho);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

}  // namespace

extern "C" {

int otoo_sph_density(const otoo_dev_system* sys, const float* h, double* rho, const otoo_tune* tune, void* stream)
{
    otoo::Range range_("otoo_sph_density");
    OTOO_REQUIRE(sys && h && rho && tune, OTOO_EINVAL, "otoo_sph_density: NULL argument");
    OTOO_REQUIRE(sys->src && sys->groups && sys->list && sys->items && sys->counter && sys->split, OTOO_EINVAL,
                 "otoo_sph_density: NULL device array");
    OTOO_REQUIRE(sys->n_part >= 1 && sys->n_groups >= 1 && sys->n_items >= 0 && sys->n_crit_max >= 1, OTOO_EINVAL,
                 "otoo_sph_density: bad sizes");
    OTOO_REQUIRE(sys->n_splits == 0 || (sys->splits && sys->partial), OTOO_EINVAL,
                 "otoo_sph_density: split lists need splits and partial");
    const int ib = tune->iblock;
    OTOO_REQUIRE(ib == 1 || ib == 2 || ib == 4, OTOO_EINVAL, "otoo_sph_density: iblock must be 1, 2 or 4");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float* ht = static_cast<float*>(sys->split);
    CUDA_TRY(cudaMemsetAsync(sys->counter, 0, 2 * sizeof(uint32_t), s));
    k_h_tree<<<(unsigned)((sys->n_part + 255) / 256), 256, 0, s>>>(h, sys->perm, sys->n_part, ht, sys->counter + 1);
    CUDA_TRY(cudaGetLastError());
    if (sys->n_items > 0) {
        const int r = ib == 1 ? launch<1>(sys, ht, rho, s) : ib == 2 ? launch<2>(sys, ht, rho, s) : launch<4>(sys, ht, rho, s);
        if (r) return r;
    }
    if (sys->n_splits > 0) {
        k_density_merge<<<(unsigned)((sys->n_splits * 32 + 127) / 128), 128, 0, s>>>(*sys, rho);
        CUDA_TRY(cudaGetLastError());
    }
    return OTOO_OK;
}

int otoo_sph_direct(const otoo_src* src, const float* h, int64_t n, const int64_t* targets, int64_t n_tgt, double* rho,
                    uint32_t* status, void* stream)
{
    OTOO_REQUIRE(src && h && targets && rho && status, OTOO_EINVAL, "otoo_sph_direct: NULL pointer");
    OTOO_REQUIRE(n >= 1 && n_tgt >= 1 && n_tgt <= ((int64_t)1 << 31), OTOO_EINVAL, "otoo_sph_direct: bad sizes");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(uint32_t), s));
    k_sph_direct<<<(unsigned)((n_tgt + 127) / 128), 128, 0, s>>>(src, h, n, targets, n_tgt, rho, status);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

}  // extern "C"
