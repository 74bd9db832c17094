// SPH density on the device (Section II, "Bounding Radius for SPH"):
// rho_i = sum_j m_j W(|x_i - x_j|, h_j) (Eq. SPH_SUM with A = m) over the
// particle lists of the SPH walk (Eq. SPH_RAD), which hold every source j
// whose support can reach a particle of the group.  Readings: the M4 cubic
// spline with support radius h, the scatter form (each source's own h_j), the
// source itself included.
//
// Kernels
//   k_sph_prep        once per step, per source in tree order: its position
//                     as a float pair (hi = x rounded to FP32, lo = the
//                     remainder), m_j 8/(pi h_j^3) and 1/h_j (h through the
//                     permutation): the step's only FP64 work, as in the
//                     force step's float-pair split.
//   k_density<IB>     one work item (group, target chunk, list chunk) per warp
//                     from an atomic ticket, IB targets per lane in lane
//                     subsets that share out the kept entries of a tile (as
//                     the force kernels do); 32-entry tiles staged in shared
//                     memory as (x_j - c, m_j 8/(pi h_j^3), 1/h_j) in FP32
//                     relative to the group centre c ((hi - c) + lo), keeping
//                     only entries within (1 + 2^-10) h_j of the item's own
//                     target box (the others have W = 0 at every target; the
//                     walk's lists are cut at cell level and hold about 12
//                     times more entries than neighbours); kept entries wait
//                     in shared memory until 32 are there; each lane sums IB
//                     targets over pairs of waiting entries with packed FP32
//                     (f32x2) arithmetic and the spline as truncated powers
//                     (no branch), plain FP32 within a batch,
//                     Kahan-compensated FP32 across batches and lane subsets
//                     (pairwise, in a fixed order), FP64 output.
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
constexpr uint32_t kBadItem = 1u;   // same status bits as the force step
constexpr uint32_t kBadIndex = 2u;
constexpr float kNorm = 2.546479089470325f;  // 8 / pi

#include "pair.cuh"

// Per tree-order source k: out[2k] = (hi_x, hi_y, hi_z, m 8/(pi h^3)),
// out[2k + 1] = (lo_x, lo_y, lo_z, 1/h), h = h[perm[k]].
__global__ void k_sph_prep(const otoo_src* __restrict__ src, const float* __restrict__ h,
                           const int64_t* __restrict__ perm, int64_t n, float4* __restrict__ out,
                           uint32_t* __restrict__ status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = perm ? perm[k] : k;
    float hk = 1.0f;
    if (i < 0 || i >= n) {
        atomicOr(status, kBadIndex);
    } else {
        hk = h[i];
    }
    const otoo_src s = src[k];
    const float ih = 1.0f / hk;
    const float hx = __double2float_rn(s.x), hy = __double2float_rn(s.y), hz = __double2float_rn(s.z);
    out[2 * k] = make_float4(hx, hy, hz, s.m * kNorm * ih * ih * ih);
    out[2 * k + 1] = make_float4(__double2float_rn(s.x - (double)hx), __double2float_rn(s.y - (double)hy),
                                 __double2float_rn(s.z - (double)hz), ih);
}

// Square roots of both halves of a float pair (the hardware approximation,
// PTX sqrt.approx.ftz.f32, relative error about 2^-23; sqrt(0) = 0).
__device__ __forceinline__ f2 f2sqrt(f2 a)
{
    float lo, hi;
    f2unpack(a, lo, hi);
    asm("sqrt.approx.ftz.f32 %0, %0;" : "+f"(lo));
    asm("sqrt.approx.ftz.f32 %0, %0;" : "+f"(hi));
    return f2pack(lo, hi);
}

// M4 cubic spline shape of both halves, q = r / h >= 0, as truncated powers:
// w(q) = 2 max(1 - q, 0)^3 - max(1 - 2q, 0)^3, which is 1 - 6q^2 + 6q^3 for
// q <= 1/2, 2 (1 - q)^3 for 1/2 <= q <= 1 and 0 beyond (no branch: the two
// clamps are the only scalar steps).
__device__ __forceinline__ f2 f2w_m4(f2 q)
{
    const f2 one = f2pack(1.f, 1.f), mone = f2pack(-1.f, -1.f), two = f2pack(2.f, 2.f);
    float s0, s1, t0, t1;
    f2unpack(f2fma(q, mone, one), s0, s1);  // 1 - q
    f2unpack(f2fma(q, two, mone), t0, t1);  // -(1 - 2q)
    const f2 s = f2pack(fmaxf(s0, 0.f), fmaxf(s1, 0.f));
    const f2 t = f2pack(fminf(t0, 0.f), fminf(t1, 0.f));
    return f2fma(f2mul(f2mul(s, s), s), two, f2mul(f2mul(t, t), t));
}

// Partial slots [slot0, slot0 + n) lie inside sys.partial.
__device__ __forceinline__ bool sph_slots_fit(const otoo_dev_system& sys, int64_t slot0, int64_t n)
{
    return slot0 >= 0 && n >= 0 && (slot0 + n) * sys.n_crit_max * 4 <= sys.partial_doubles;
}

template <int IB>
__global__ void __launch_bounds__(kDW * 32) k_density(otoo_dev_system sys, const float4* __restrict__ rec,
                                                      double* __restrict__ rho)
{
    // kept entries waiting (up to 31 plus a tile's 32), one row per field:
    // x, y, z relative to the group centre, m 8/(pi h^3), 1/h; entries 2m and
    // 2m + 1 of a row load as one float pair
    __shared__ __align__(16) float tq[kDW][5][64];
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
                 (it.slot < 0 || (g.count <= sys.n_crit_max && sph_slots_fit(sys, it.slot, 1)));
        }
        if (!ok) {
            if (lane == 0) atomicOr(counter + 1, kBadItem);
            continue;
        }
        // the item's targets, IB per lane in nsub lane subsets of P lanes;
        // subset js takes every nsub-th kept entry of a tile
        const int P = (it.ni + IB - 1) / IB;
        const int nsub = 32 / P;
        const int islot = lane % P, js = lane / P;
        const bool active = js < nsub;
        const float cx = __double2float_rn(g.cx), cy = __double2float_rn(g.cy), cz = __double2float_rn(g.cz);
        float xi[IB], yi[IB], zi[IB];
        float as[IB], ac[IB];  // Kahan sum of the lane's share: as - ac
        float blo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, bhi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
#pragma unroll
        for (int r = 0; r < IB; ++r) {
            const int k = islot + r * P;
            as[r] = ac[r] = 0.f;
            xi[r] = yi[r] = zi[r] = 0.f;
            if (active && k < it.ni) {
                float4 a, b;
                ld256x2(rec + 2 * ((int64_t)g.first + it.i0 + k), a, b);
                xi[r] = rel32(a.x, b.x, cx);
                yi[r] = rel32(a.y, b.y, cy);
                zi[r] = rel32(a.z, b.z, cz);
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
        f2 xi2[IB], yi2[IB], zi2[IB];
#pragma unroll
        for (int r = 0; r < IB; ++r) {
            xi2[r] = f2pack(xi[r], xi[r]);
            yi2[r] = f2pack(yi[r], yi[r]);
            zi2[r] = f2pack(zi[r], zi[r]);
        }
        // evaluates the first cnt waiting entries for the lane's targets, two
        // entries per packed operation (an odd last entry is paired with a
        // zero entry, which adds exactly nothing), and adds the batch into
        // the Kahan sums
        auto batch = [&](int cnt) {
            if (cnt & 1) {
                if (lane < 5) tq[w][lane][cnt] = 0.f;
                __syncwarp();
            }
            const int npair = (cnt + 1) >> 1;
            const f2* fx = reinterpret_cast<const f2*>(tq[w][0]);
            const f2* fy = reinterpret_cast<const f2*>(tq[w][1]);
            const f2* fz = reinterpret_cast<const f2*>(tq[w][2]);
            const f2* fm = reinterpret_cast<const f2*>(tq[w][3]);
            const f2* fh = reinterpret_cast<const f2*>(tq[w][4]);
            f2 part2[IB];
#pragma unroll
            for (int r = 0; r < IB; ++r) part2[r] = f2pack(0.f, 0.f);
            for (int m = active ? js : npair; m < npair; m += nsub) {
                const f2 px = fx[m], py = fy[m], pz = fz[m], pm = fm[m], ph = fh[m];
#pragma unroll
                for (int r = 0; r < IB; ++r) {
                    const f2 dx = f2sub(px, xi2[r]), dy = f2sub(py, yi2[r]), dz = f2sub(pz, zi2[r]);
                    const f2 r2 = f2fma(dx, dx, f2fma(dy, dy, f2mul(dz, dz)));
                    part2[r] = f2fma(pm, f2w_m4(f2mul(f2sqrt(r2), ph)), part2[r]);
                }
            }
            float part[IB];
#pragma unroll
            for (int r = 0; r < IB; ++r) {
                float lo, hi;
                f2unpack(part2[r], lo, hi);
                part[r] = lo + hi;
            }
#pragma unroll
            for (int r = 0; r < IB; ++r) {
                const float y = __fsub_rn(part[r], ac[r]);
                const float tt = __fadd_rn(as[r], y);
                ac[r] = __fsub_rn(__fsub_rn(tt, as[r]), y);
                as[r] = tt;
            }
            __syncwarp();
        };
        // list tiles of 32 entries, one per lane; each tile's indices are
        // loaded one tile ahead
        auto fetch_idx = [&](int32_t j, bool& has) -> int32_t {
            has = j + lane < it.j1;
            return has ? sys.list[g.list_off + j + lane] : 0;
        };
        bool has0;
        int32_t e0 = fetch_idx(it.j0, has0);
        int nk = 0;  // kept entries waiting in tq
        for (int32_t j = it.j0; j < it.j1; j += 32) {
            bool has1;
            const int32_t e1 = fetch_idx(j + 32, has1);
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            float ih = 0.f;
            bool keep = false;
            if (has0) {
                const int32_t e = e0;
                if (e >= 0 && e < sys.n_part) {
                    float4 a, b;
                    ld256x2(rec + 2 * (int64_t)e, a, b);
                    ih = b.w;
                    p = make_float4(rel32(a.x, b.x, cx), rel32(a.y, b.y, cy), rel32(a.z, b.z, cz), a.w);
                    // distance from the entry to the target box against its
                    // support: kept unless d >= (1 + 2^-10) h, where every
                    // target's q = r / h exceeds 1 even after rounding
                    const float dx = fmaxf(0.f, fmaxf(blo[0] - p.x, p.x - bhi[0]));
                    const float dy = fmaxf(0.f, fmaxf(blo[1] - p.y, p.y - bhi[1]));
                    const float dz = fmaxf(0.f, fmaxf(blo[2] - p.z, p.z - bhi[2]));
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    keep = d2 * ih * ih < (1.0f + 0x1p-10f) * (1.0f + 0x1p-10f);
                } else {
                    atomicOr(counter + 1, kBadIndex);
                }
            }
            const unsigned km = __ballot_sync(kFull, keep);
            if (keep) {
                const int slot = nk + __popc(km & ((1u << lane) - 1u));
                tq[w][0][slot] = p.x;
                tq[w][1][slot] = p.y;
                tq[w][2][slot] = p.z;
                tq[w][3][slot] = p.w;
                tq[w][4][slot] = ih;
            }
            nk += __popc(km);
            __syncwarp();
            if (nk >= 32) {  // a full batch: evaluate it, move the rest to the front
                batch(32);
                if (lane < nk - 32) {
#pragma unroll
                    for (int f = 0; f < 5; ++f) tq[w][f][lane] = tq[w][f][32 + lane];
                }
                nk -= 32;
                __syncwarp();
            }
            has0 = has1, e0 = e1;
        }
        if (nk > 0) batch(nk);
        // merge the lane subsets into js == 0 (pairwise, a fixed order)
        double acc[IB];
#pragma unroll
        for (int r = 0; r < IB; ++r) {
            merge_subsets(as[r], ac[r], js, nsub, P);
            acc[r] = (double)as[r] - (double)ac[r];
        }
#pragma unroll
        for (int r = 0; r < IB; ++r) {
            const int k = islot + r * P;
            if (js != 0 || k >= it.ni) continue;
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
    if (sp.g < 0 || sp.g >= sys.n_groups || sp.n_chunks < 1 || !sph_slots_fit(sys, sp.slot0, sp.n_chunks)) {
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
int launch(const otoo_dev_system* sys, const float4* rec, double* rho, cudaStream_t s)
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
    k_density<IB><<<(unsigned)blocks, kDW * 32, 0, s>>>(*sys, rec, rho);
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
    OTOO_REQUIRE(sys->n_splits == 0 || (sys->splits && sys->partial && sys->partial_doubles >= 4 * (int64_t)sys->n_crit_max),
                 OTOO_EINVAL, "otoo_sph_density: split lists need splits and partial scratch");
    const int ib = tune->iblock;
    OTOO_REQUIRE(ib == 1 || ib == 2 || ib == 4, OTOO_EINVAL, "otoo_sph_density: iblock must be 1, 2 or 4");
    OTOO_REQUIRE((reinterpret_cast<uintptr_t>(sys->split) & 31) == 0, OTOO_EINVAL,
                 "otoo_sph_density: the split scratch must be 32-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float4* rec = static_cast<float4*>(sys->split);
    CUDA_TRY(cudaMemsetAsync(sys->counter, 0, 2 * sizeof(uint32_t), s));
    k_sph_prep<<<(unsigned)((sys->n_part + 255) / 256), 256, 0, s>>>(sys->src, h, sys->perm, sys->n_part, rec,
                                                                      sys->counter + 1);
    CUDA_TRY(cudaGetLastError());
    if (sys->n_items > 0) {
        const int r = ib == 1 ? launch<1>(sys, rec, rho, s) : ib == 2 ? launch<2>(sys, rec, rho, s) : launch<4>(sys, rec, rho, s);
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
