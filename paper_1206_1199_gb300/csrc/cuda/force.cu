// Device half of the force step: every particle of a group against every
// entry of the group's shared interaction list.
//
// Paper: Section II (particle-particle and particle-cell interactions, the
// cell acting as a virtual particle at its centre of mass), Section III-D
// (the GPU evaluates the interactions of a group that shares one walk).  The
// quadrupole cell term, the FP32 centre-relative arithmetic with per-thread
// Kahan sums, the persistent load-balanced launch and the CUDA graph are this
// library's design for sm_103a; the pair law with Plummer softening is a
// reading (the paper keeps a softening length per particle but does not print
// the law).
//
// Kernels of one step (recorded into a CUDA graph):
//   k_split       FP32 form only: each source position as a float pair
//                 (hi, lo), once per step -- the FP64 work of the step.
//   k_force_warp  FP32 form: one work item per warp, no block-wide barrier;
//                 FP32 pairs on group-centre-relative coordinates, plain FP32
//                 sums between Kahan-compensated flushes, FP64 merge of the
//                 lane-level j-split and FP64 outputs.
//   k_force_f64   FP64 form (comparison form): one work item per CTA, every
//                 pair in FP64.
//   k_merge       FP64 sum of the chunk partials of split lists, in chunk
//                 order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../common.h"

using namespace otoo;

namespace {

// Status bits written to counter[1].
constexpr uint32_t kBadItem = 1u;
constexpr uint32_t kBadIndex = 2u;

#include "pair.cuh"

__device__ __forceinline__ void load_src(const otoo_src* src, int64_t idx, double& x, double& y, double& z, float& m)
{
    const double2* p = reinterpret_cast<const double2*>(src + idx);
    const double2 a = __ldg(p);
    const double2 b = __ldg(p + 1);
    x = a.x;
    y = a.y;
    z = b.x;
    m = __int_as_float((int)(__double_as_longlong(b.y) & 0xffffffffll));
}

// Partial slots [slot0, slot0 + n) lie inside sys.partial (each slot holds
// n_crit_max targets of 4 doubles).
__device__ __forceinline__ bool slots_fit(const otoo_dev_system& sys, int64_t slot0, int64_t n)
{
    return slot0 >= 0 && n >= 0 && (slot0 + n) * sys.n_crit_max * 4 <= sys.partial_doubles;
}

// Checks an item against the system's sizes; fills grp.
__device__ __forceinline__ bool item_ok(const otoo_dev_system& sys, const otoo_item& item, otoo_group& grp, int max_ni)
{
    if (item.g < 0 || item.g >= sys.n_groups) return false;
    grp = sys.groups[item.g];
    const int64_t L = (int64_t)grp.n_cell + grp.n_part;
    return grp.count >= 1 && grp.first >= 0 && (int64_t)grp.first + grp.count <= sys.n_part && grp.n_cell >= 0 &&
           grp.n_part >= 0 && item.ni >= 1 && item.ni <= max_ni && item.i0 >= 0 &&
           (int64_t)item.i0 + item.ni <= grp.count && item.j0 >= 0 && item.j0 <= item.j1 && item.j1 <= L &&
           grp.list_off >= 0 && grp.list_off + L <= sys.n_list &&
           (item.slot < 0 || (grp.count <= sys.n_crit_max && slots_fit(sys, item.slot, 1)));
}

// Final write of one target: the output, or the FP64 partial of the item's
// list chunk.  The kernels take the self pair (r = 0, which adds -m_i / eps
// to phi_i) out of the item whose list chunk starts at entry 0.
__device__ __forceinline__ void write_target(const otoo_dev_system& sys, const otoo_group& grp, const otoo_item& item,
                                             int i, const double a[4], double* __restrict__ accel,
                                             double* __restrict__ pot)
{
    const int ig = item.i0 + i;
    if (item.slot < 0) {
        const int64_t t = (int64_t)grp.first + ig;
        const int64_t o = sys.perm ? sys.perm[t] : t;
        accel[3 * o] = a[0];
        accel[3 * o + 1] = a[1];
        accel[3 * o + 2] = a[2];
        pot[o] = a[3];
    } else {
        double* dst = sys.partial + ((int64_t)item.slot * sys.n_crit_max + ig) * 4;
        dst[0] = a[0];
        dst[1] = a[1];
        dst[2] = a[2];
        dst[3] = a[3];
    }
}

// Position split for the FP32 form, once per step: hi = x rounded to FP32,
// lo = (x - hi) rounded to FP32.  A centre-relative coordinate is then
// (hi - c) + lo in FP32 with c an FP32 value: hi - c is exact for every entry
// within a factor of two of c (Sterbenz), so near entries keep the accuracy of
// an FP64 subtraction rounded once to FP32, and far entries stay within about
// one FP32 ulp of it.
__global__ void k_split(const otoo_src* __restrict__ src, float4* __restrict__ out, int64_t n)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double x, y, z;
    float m;
    load_src(src, s, x, y, z, m);
    const float hx = __double2float_rn(x), hy = __double2float_rn(y), hz = __double2float_rn(z);
    out[2 * s] = make_float4(hx, hy, hz, m);
    out[2 * s + 1] = make_float4(__double2float_rn(x - (double)hx), __double2float_rn(y - (double)hy),
                                 __double2float_rn(z - (double)hz), 0.f);
}

// Centre-relative coordinates of n sources as the FP32 force kernels stage
// them (otoo_centre_relative): rel32 of each float pair written by k_split.
__global__ void k_centre_relative(const float4* __restrict__ pairs, int64_t n, float cx, float cy, float cz,
                                  float* __restrict__ out)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float4 h = pairs[2 * s], l = pairs[2 * s + 1];
    out[3 * s] = rel32(h.x, l.x, cx);
    out[3 * s + 1] = rel32(h.y, l.y, cy);
    out[3 * s + 2] = rel32(h.z, l.z, cz);
}

#include "force_warp.cuh"
#include "force_warp2.cuh"

// FP64 form: one work item per CTA of B threads, IB targets per thread,
// B entries staged per tile, every pair in FP64.
template <int B, int IB>
__global__ void __launch_bounds__(B) k_force_f64(const otoo_dev_system sys, double* __restrict__ accel,
                                                 double* __restrict__ pot)
{
    __shared__ V4<double> s_src[B];
    __shared__ V4<double> s_qa[B];
    __shared__ V4<double> s_qb[B];
    __shared__ double s_red[B * IB * 4];
    __shared__ int s_ticket;

    const int tid = threadIdx.x;
    uint32_t* status = sys.counter + 1;
    const bool has_quad = sys.quad != nullptr;

    for (;;) {
        if (tid == 0) s_ticket = (int)atomicAdd(sys.counter, 1u);
        __syncthreads();
        const int it = s_ticket;
        __syncthreads();
        if (it >= sys.n_items) break;

        const otoo_item item = sys.items[it];
        otoo_group grp;
        if (!item_ok(sys, item, grp, B * IB)) {
            if (tid == 0) atomicOr(status, kBadItem);
            continue;
        }
        const int ni = item.ni;
        const int P = (ni + IB - 1) / IB;
        const int nsplit = B / P;
        const int islot = tid % P, js = tid / P;
        const bool active = js < nsplit;
        const double eps2 = grp.eps2;
        const double cx = grp.cx, cy = grp.cy, cz = grp.cz;

        double xi[IB], yi[IB], zi[IB];
        Acc<double> acc[IB];
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            const int i = islot + k * P;
            xi[k] = yi[k] = zi[k] = 0.0;
            if (active && i < ni) {
                double x, y, z;
                float m;
                load_src(sys.src, (int64_t)grp.first + item.i0 + i, x, y, z, m);
                xi[k] = x - cx;
                yi[k] = y - cy;
                zi[k] = z - cz;
            }
            acc[k].zero();
        }

        const int32_t* lst = sys.list + grp.list_off;
        for (int seg = 0; seg < 2; ++seg) {
            const bool is_cell = seg == 0;
            const int s0 = is_cell ? item.j0 : max(item.j0, grp.n_cell);
            const int s1 = is_cell ? min(item.j1, grp.n_cell) : item.j1;
            const bool quad = is_cell && has_quad;
            for (int base = s0; base < s1; base += B) {
                const int cnt = min(B, s1 - base);
                if (tid < cnt) {
                    const int idx = __ldg(lst + base + tid);
                    const bool good = is_cell ? (idx >= sys.n_part && idx < sys.n_src) : (idx >= 0 && idx < sys.n_part);
                    V4<double> v = {0, 0, 0, 0};
                    if (good) {
                        double x, y, z;
                        float m;
                        load_src(sys.src, idx, x, y, z, m);
                        v = V4<double>{x - cx, y - cy, z - cz, (double)m};
                    } else {
                        atomicOr(status, kBadIndex);
                    }
                    s_src[tid] = v;
                    if (quad) {
                        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                        if (good) {
                            const float4* qp = reinterpret_cast<const float4*>(sys.quad + (idx - sys.n_part));
                            a = __ldg(qp);
                            b = __ldg(qp + 1);
                        }
                        s_qa[tid] = V4<double>{a.x, a.y, a.z, a.w};
                        // (xz, yz, B_2 eps^2, -) for the softened quadrupole term
                        s_qb[tid] = V4<double>{b.x, b.y, (double)b.z * eps2, 0.0};
                    }
                }
                __syncthreads();
                if (active) {
                    double p[IB][4];
#pragma unroll
                    for (int k = 0; k < IB; ++k) p[k][0] = p[k][1] = p[k][2] = p[k][3] = 0.0;
                    if (quad) {
                        for (int j = js; j < cnt; j += nsplit) {
                            const V4<double> s = s_src[j];
                            const V4<double> qa = s_qa[j];
                            const V4<double> qb = s_qb[j];
#pragma unroll
                            for (int k = 0; k < IB; ++k) pair_quad(s, qa, qb, xi[k], yi[k], zi[k], eps2, p[k]);
                        }
                    } else {
                        for (int j = js; j < cnt; j += nsplit) {
                            const V4<double> s = s_src[j];
#pragma unroll
                            for (int k = 0; k < IB; ++k) pair_mono(s, xi[k], yi[k], zi[k], eps2, p[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < IB; ++k) acc[k].add(p[k]);
                }
                __syncthreads();
            }
        }

        if (active) {
#pragma unroll
            for (int k = 0; k < IB; ++k)
#pragma unroll
                for (int c = 0; c < 4; ++c) s_red[((js * P + islot) * IB + k) * 4 + c] = acc[k].value(c);
        }
        __syncthreads();
        for (int i = tid; i < ni; i += B) {
            const int sl = i % P, k = i / P;
            double a[4] = {0, 0, 0, 0};
            for (int j = 0; j < nsplit; ++j)
#pragma unroll
                for (int c = 0; c < 4; ++c) a[c] += s_red[((j * P + sl) * IB + k) * 4 + c];
            if (item.j0 == 0) {
                // the self pair added -m_i rsqrt(eps^2) in FP64: take it out
                double x, y, z;
                float m;
                load_src(sys.src, (int64_t)grp.first + item.i0 + i, x, y, z, m);
                a[3] += (double)m * rsqrt(eps2);
            }
            write_target(sys, grp, item, i, a, accel, pot);
        }
        __syncthreads();
    }
}

// Sum the chunk partials of each split list in chunk order (one warp per list).
__global__ void k_merge(const otoo_dev_system sys, double* __restrict__ accel, double* __restrict__ pot)
{
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= sys.n_splits) return;
    const otoo_split sp = sys.splits[w];
    bool ok = sp.g >= 0 && sp.g < sys.n_groups && sp.n_chunks >= 1 && slots_fit(sys, sp.slot0, sp.n_chunks);
    otoo_group grp;
    if (ok) {
        grp = sys.groups[sp.g];
        ok = grp.count >= 1 && grp.count <= sys.n_crit_max && grp.first >= 0 &&
             (int64_t)grp.first + grp.count <= sys.n_part;
    }
    if (!ok) {
        if (lane == 0) atomicOr(sys.counter + 1, kBadItem);
        return;
    }
    for (int i = lane; i < grp.count; i += 32) {
        double a[4] = {0, 0, 0, 0};
        for (int c = 0; c < sp.n_chunks; ++c) {
            const double* s = sys.partial + ((int64_t)(sp.slot0 + c) * sys.n_crit_max + i) * 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] += s[k];
        }
        const int64_t t = (int64_t)grp.first + i;
        const int64_t o = sys.perm ? sys.perm[t] : t;
        accel[3 * o] = a[0];
        accel[3 * o + 1] = a[1];
        accel[3 * o + 2] = a[2];
        pot[o] = a[3];
    }
}

// ---------------------------------------------------------------------------
// host side: kernel choice, launch shape, CUDA graph cache

using Kernel = void (*)(const otoo_dev_system, double*, double*);

Kernel pick_f32(int B, int IB, int tile, int packed)
{
    const int spl = tile / 32;
#define PICK(NW_, IB_, SPL_) \
    if (B == NW_ * 32 && IB == IB_ && spl == SPL_) return k_force_warp<NW_, IB_, SPL_>;
#define PICK2(NW_, IB_, SPL_) \
    if (B == NW_ * 32 && IB == IB_ && spl == SPL_) return k_force_warp2<NW_, IB_, SPL_>;
    if (packed) {
        PICK2(4, 1, 4) PICK2(4, 2, 4) PICK2(4, 2, 8) PICK2(2, 2, 4) PICK2(2, 1, 4) PICK2(4, 1, 8)
        return nullptr;
    }
    PICK(4, 1, 4) PICK(4, 2, 2) PICK(4, 2, 4) PICK(4, 2, 8) PICK(4, 4, 4) PICK(4, 4, 8)
    PICK(2, 2, 4) PICK(2, 4, 4) PICK(8, 2, 4) PICK(8, 1, 4)
#undef PICK
#undef PICK2
    return nullptr;
}

// FP64 form: B threads per CTA for a plan made with iblock targets per lane
// (items of at most 32 * iblock targets).
Kernel pick_f64(int IB)
{
    if (IB == 1) return k_force_f64<128, 1>;
    if (IB == 2) return k_force_f64<128, 2>;
    return k_force_f64<128, 4>;
}

int check_tune(const otoo_tune* t)
{
    OTOO_REQUIRE(t, OTOO_EINVAL, "tune is NULL");
    OTOO_REQUIRE(pick_f32(t->block, t->iblock, t->tile, t->packed) != nullptr, OTOO_EINVAL,
                 "unsupported tune: block %d, iblock %d, tile %d", t->block, t->iblock, t->tile);
    OTOO_REQUIRE(t->split >= 32, OTOO_EINVAL, "split must be >= 32");
    OTOO_REQUIRE(t->ctas_per_sm >= 0 && t->ctas_per_sm <= 32, OTOO_EINVAL, "ctas_per_sm out of range");
    return OTOO_OK;
}

#define CUDA_TRY(expr)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return set_error(OTOO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

// Copies the work ticket and status word (counter[0..1], device) out on
// stream, synchronises it and turns the status bits into an error code.
int read_status(const uint32_t* counter, void* stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t h[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(h, counter, sizeof(h), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (h[1] & kBadItem) return set_error(OTOO_EDEVICE, "a work item, split or group failed its bounds check");
    if (h[1] & kBadIndex) return set_error(OTOO_EDEVICE, "a list entry indexed outside its source range");
    return OTOO_OK;
}

// Records the launches of one force step on stream s.
}  // namespace

int otoo::enqueue_split(const otoo_src* src, float* out, int64_t n, void* stream)
{
    if (n <= 0) return OTOO_OK;
    const int64_t nb = (n + 255) / 256;
    k_split<<<(unsigned)nb, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(src, reinterpret_cast<float4*>(out), n);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

namespace {

int enqueue_force(const otoo_dev_system* sys, double* accel, double* pot, int precision, const otoo_tune* t,
                  cudaStream_t s)
{
    const bool fp64 = precision == OTOO_FP64;
    Kernel fn = fp64 ? pick_f64(t->iblock) : pick_f32(t->block, t->iblock, t->tile, t->packed);
    const int block = fp64 ? 128 : t->block;
    int dev = 0, nsm = 0, occ = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, 0));
    if (occ < 1) return set_error(OTOO_EINVAL, "force kernel does not fit on an SM");
    const int per_sm = t->ctas_per_sm > 0 ? std::min(t->ctas_per_sm, occ) : occ;
    const int64_t units = fp64 ? sys->n_items : ((int64_t)sys->n_items + block / 32 - 1) / (block / 32);
    const int grid = (int)std::min<int64_t>(units, (int64_t)nsm * per_sm);
    CUDA_TRY(cudaMemsetAsync(sys->counter, 0, 2 * sizeof(uint32_t), s));
    if (!fp64) {
        const int64_t nb = (sys->n_src + 255) / 256;
        k_split<<<(unsigned)nb, 256, 0, s>>>(sys->src, reinterpret_cast<float4*>(sys->split), sys->n_src);
        CUDA_TRY(cudaGetLastError());
    }
    if (grid > 0) {
        fn<<<grid, block, 0, s>>>(*sys, accel, pot);
        CUDA_TRY(cudaGetLastError());
    }
    if (sys->n_splits > 0) {
        k_merge<<<(sys->n_splits + 3) / 4, 128, 0, s>>>(*sys, accel, pot);
        CUDA_TRY(cudaGetLastError());
    }
    return OTOO_OK;
}

struct GraphKey {
    otoo_dev_system sys;
    double* accel;
    double* pot;
    int precision, device;
    otoo_tune tune;
    bool operator==(const GraphKey& o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec;
    uint64_t last_use;
};

std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
uint64_t g_graph_clock = 0;
constexpr size_t kMaxGraphs = 16;

int validate_sys(const otoo_dev_system* sys)
{
    OTOO_REQUIRE(sys, OTOO_EINVAL, "sys is NULL");
    OTOO_REQUIRE(sys->n_part >= 1 && sys->n_src >= sys->n_part && sys->n_src <= INT32_MAX, OTOO_EINVAL,
                 "bad sizes n_part %lld n_src %lld", (long long)sys->n_part, (long long)sys->n_src);
    OTOO_REQUIRE(sys->n_groups >= 1 && sys->n_items >= 0 && sys->n_splits >= 0 && sys->n_list >= 0, OTOO_EINVAL,
                 "bad counts");
    OTOO_REQUIRE(sys->n_crit_max >= 1 && sys->n_crit_max <= kMaxGroup, OTOO_EINVAL, "n_crit_max out of range");
    OTOO_REQUIRE(sys->src && sys->groups && sys->counter && (sys->n_items == 0 || (sys->items && sys->list)),
                 OTOO_EINVAL, "NULL device array");
    OTOO_REQUIRE(sys->partial_doubles >= 0, OTOO_EINVAL, "partial_doubles < 0");
    OTOO_REQUIRE(sys->n_splits == 0 ||
                     (sys->splits && sys->partial && sys->partial_doubles >= 4 * (int64_t)sys->n_crit_max),
                 OTOO_EINVAL, "split lists need partial scratch (at least 4 * n_crit_max doubles)");
    OTOO_REQUIRE((reinterpret_cast<uintptr_t>(sys->quad) & 31) == 0 && (reinterpret_cast<uintptr_t>(sys->split) & 31) == 0,
                 OTOO_EINVAL, "quad and split must be 32-byte aligned (one 32-byte load per record)");
    return OTOO_OK;
}

}  // namespace

extern "C" {

int otoo_force(const otoo_dev_system* sys, double* accel, double* pot, int32_t precision, const otoo_tune* tune,
               void* stream)
{
    otoo::Range range_("otoo_force");
    int rc = validate_sys(sys);
    if (rc) return rc;
    OTOO_REQUIRE(accel && pot, OTOO_EINVAL, "accel/pot is NULL");
    OTOO_REQUIRE(precision == OTOO_FP32K || precision == OTOO_FP64, OTOO_EINVAL, "bad precision %d", precision);
    rc = check_tune(tune);
    if (rc) return rc;
    OTOO_REQUIRE(precision == OTOO_FP64 || sys->split != nullptr, OTOO_EINVAL,
                 "OTOO_FP32K needs the split scratch (32 bytes per source)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.sys = *sys;
    key.accel = accel;
    key.pot = pot;
    key.precision = precision;
    CUDA_TRY(cudaGetDevice(&key.device));
    key.tune = *tune;
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (GraphEntry& e : g_graphs) {
        if (e.key == key) {
            e.last_use = ++g_graph_clock;
            CUDA_TRY(cudaGraphLaunch(e.exec, s));
            return OTOO_OK;
        }
    }
    // record the step into a graph on a private stream
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {
        cudaStreamDestroy(cs);
        return set_error(OTOO_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(ce));
    }
    rc = enqueue_force(sys, accel, pot, precision, tune, cs);
    ce = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess) return set_error(OTOO_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
    cudaGraphExec_t exec;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return set_error(OTOO_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ce));
    if (g_graphs.size() >= kMaxGraphs) {
        size_t old = 0;
        for (size_t k = 1; k < g_graphs.size(); ++k)
            if (g_graphs[k].last_use < g_graphs[old].last_use) old = k;
        cudaGraphExecDestroy(g_graphs[old].exec);
        g_graphs.erase(g_graphs.begin() + old);
    }
    g_graphs.push_back(GraphEntry{key, exec, ++g_graph_clock});
    CUDA_TRY(cudaGraphLaunch(exec, s));
    return OTOO_OK;
}

int otoo_check_status(const otoo_dev_system* sys, void* stream)
{
    OTOO_REQUIRE(sys && sys->counter, OTOO_EINVAL, "sys/counter is NULL");
    return read_status(sys->counter, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// otoo_force_host: host arrays in, host arrays out (device buffers cached)

namespace {

constexpr int kHostBufs = 10;
struct HostPathBuffers {
    int device = -1;
    void* p[kHostBufs] = {nullptr};
    size_t cap[kHostBufs] = {0};
};
std::mutex g_host_mu;
HostPathBuffers g_host;

int ensure(int k, size_t bytes)
{
    if (g_host.cap[k] >= bytes && g_host.p[k]) return OTOO_OK;
    if (g_host.p[k]) cudaFree(g_host.p[k]);
    g_host.p[k] = nullptr;
    g_host.cap[k] = 0;
    const size_t b = std::max<size_t>(bytes, 256);
    CUDA_TRY(cudaMalloc(&g_host.p[k], b));
    g_host.cap[k] = b;
    return OTOO_OK;
}

}  // namespace

extern "C" int otoo_centre_relative(const otoo_src* src, int64_t n, const double* c, float* out, void* scratch,
                                    void* stream)
{
    OTOO_REQUIRE(src && c && out && scratch, OTOO_EINVAL, "otoo_centre_relative: NULL pointer");
    OTOO_REQUIRE(n >= 1 && n <= INT32_MAX, OTOO_EINVAL, "otoo_centre_relative: bad n");
    OTOO_REQUIRE((reinterpret_cast<uintptr_t>(scratch) & 31) == 0, OTOO_EINVAL,
                 "otoo_centre_relative: scratch must be 32-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float4* pairs = static_cast<float4*>(scratch);
    const unsigned nb = (unsigned)((n + 255) / 256);
    k_split<<<nb, 256, 0, s>>>(src, pairs, n);
    CUDA_TRY(cudaGetLastError());
    k_centre_relative<<<nb, 256, 0, s>>>(pairs, n, (float)c[0], (float)c[1], (float)c[2], out);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

namespace {
// The device address of pinned (page-locked) host memory, or NULL for any
// other pointer (pageable memory, device memory, an unknown address).
double* pinned_device_address(double* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the error of an unknown pointer
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? static_cast<double*>(at.devicePointer) : nullptr;
}
}  // namespace

extern "C" int otoo_force_host(const otoo_lists_view* lv, const otoo_plan_info* pl, double* accel, double* pot,
                               int32_t precision, const otoo_tune* tune, void* stream)
{
    otoo::Range range_("otoo_force_host");
    OTOO_REQUIRE(lv && pl && accel && pot, OTOO_EINVAL, "otoo_force_host: NULL argument");
    OTOO_REQUIRE(lv->n_part >= 1 && lv->n_groups >= 1, OTOO_EINVAL, "otoo_force_host: empty input");
    std::lock_guard<std::mutex> lock(g_host_mu);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (g_host.device != dev) {
        // buffers of a previous device are left to that device's context
        for (int k = 0; k < kHostBufs; ++k) g_host.p[k] = nullptr, g_host.cap[k] = 0;
        g_host.device = dev;
    }
    const int64_t nc = lv->n_src - lv->n_part;
    const size_t bytes[kHostBufs] = {sizeof(otoo_src) * (size_t)lv->n_src,
                                     sizeof(otoo_quad) * (size_t)std::max<int64_t>(nc, 1),
                                     sizeof(otoo_group) * (size_t)lv->n_groups,
                                     sizeof(int32_t) * (size_t)std::max<int64_t>(lv->n_list, 1),
                                     sizeof(otoo_item) * (size_t)std::max<int64_t>(pl->n_items, 1),
                                     sizeof(otoo_split) * (size_t)std::max<int64_t>(pl->n_splits, 1),
                                     sizeof(int64_t) * (size_t)lv->n_part,
                                     sizeof(double) * (size_t)(std::max<int64_t>(pl->partial_doubles, 1) + 4 * lv->n_part),
                                     sizeof(uint32_t) * 4,
                                     32 * (size_t)lv->n_src};
    for (int k = 0; k < kHostBufs; ++k) {
        int rc = ensure(k, bytes[k]);
        if (rc) return rc;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemcpyAsync(g_host.p[0], lv->src, bytes[0], cudaMemcpyHostToDevice, s));
    if (lv->use_quad && nc > 0) CUDA_TRY(cudaMemcpyAsync(g_host.p[1], lv->quad, bytes[1], cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(g_host.p[2], lv->groups, bytes[2], cudaMemcpyHostToDevice, s));
    if (lv->n_list > 0) CUDA_TRY(cudaMemcpyAsync(g_host.p[3], lv->list, bytes[3], cudaMemcpyHostToDevice, s));
    if (pl->n_items > 0) CUDA_TRY(cudaMemcpyAsync(g_host.p[4], pl->items, bytes[4], cudaMemcpyHostToDevice, s));
    if (pl->n_splits > 0) CUDA_TRY(cudaMemcpyAsync(g_host.p[5], pl->splits, bytes[5], cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(g_host.p[6], lv->perm, bytes[6], cudaMemcpyHostToDevice, s));
    otoo_dev_system sys;
    std::memset(&sys, 0, sizeof(sys));
    sys.n_part = lv->n_part;
    sys.n_src = lv->n_src;
    sys.n_list = lv->n_list;
    sys.n_groups = (int32_t)lv->n_groups;
    sys.n_items = (int32_t)pl->n_items;
    sys.n_splits = (int32_t)pl->n_splits;
    sys.n_crit_max = pl->n_crit_max;
    sys.src = (const otoo_src*)g_host.p[0];
    sys.quad = lv->use_quad ? (const otoo_quad*)g_host.p[1] : nullptr;
    sys.groups = (const otoo_group*)g_host.p[2];
    sys.list = (const int32_t*)g_host.p[3];
    sys.items = (const otoo_item*)g_host.p[4];
    sys.splits = (const otoo_split*)g_host.p[5];
    sys.perm = (const int64_t*)g_host.p[6];
    double* out = (double*)g_host.p[7];
    sys.partial = out + 4 * lv->n_part;
    sys.partial_doubles = std::max<int64_t>(pl->partial_doubles, 1);
    sys.counter = (uint32_t*)g_host.p[8];
    sys.split = g_host.p[9];
    // pinned outputs: the kernel writes them in place (no copy after it)
    double* dacc = pinned_device_address(accel);
    double* dpot = pinned_device_address(pot);
    if (dacc && dpot) {
        int rc = otoo_force(&sys, dacc, dpot, precision, tune, stream);
        if (rc) return rc;
        return otoo_check_status(&sys, stream);
    }
    int rc = otoo_force(&sys, out, out + 3 * lv->n_part, precision, tune, stream);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(accel, out, sizeof(double) * 3 * (size_t)lv->n_part, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(pot, out + 3 * lv->n_part, sizeof(double) * (size_t)lv->n_part, cudaMemcpyDeviceToHost, s));
    return otoo_check_status(&sys, stream);
}

// ---------------------------------------------------------------------------
// otoo_force_static: the force step with its scratch in a library-held device
// array, for callers that cannot allocate device memory themselves.

namespace {

// Scratch of otoo_force_static: the work ticket and status word, the per-step
// float pairs of the FP32 form and the chunk partials of split lists.  Every
// GPU that loads the library holds this array until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxStaticDevices] = {nullptr};

// Device address of the array on the current device, looked up once per
// device (the symbol's host-side name is not a device address).
int static_scratch_ptr(void** out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    OTOO_REQUIRE(dev >= 0 && dev < kMaxStaticDevices, OTOO_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        OTOO_REQUIRE(p != nullptr, OTOO_ECUDA, "cudaGetSymbolAddress returned NULL");
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return OTOO_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int64_t otoo_force_static_capacity(void) { return (int64_t)kStaticScratchBytes; }

extern "C" int otoo_force_static(const otoo_dev_system* sys, int64_t partial_doubles, double* accel, double* pot,
                                 int32_t precision, const otoo_tune* tune, void* stream)
{
    otoo::Range range_("otoo_force_static");
    OTOO_REQUIRE(sys, OTOO_EINVAL, "sys is NULL");
    OTOO_REQUIRE(accel && pot, OTOO_EINVAL, "accel/pot is NULL");
    OTOO_REQUIRE(precision == OTOO_FP32K || precision == OTOO_FP64, OTOO_EINVAL, "bad precision %d", precision);
    OTOO_REQUIRE(partial_doubles >= 0, OTOO_EINVAL, "partial_doubles < 0");
    OTOO_REQUIRE(sys->n_src >= 0 && sys->n_src <= INT32_MAX, OTOO_EINVAL, "bad n_src");
    const size_t need_counter = 256;
    const size_t need_split = precision == OTOO_FP32K ? round256(32 * (size_t)sys->n_src) : 0;
    const size_t need_partial = round256(sizeof(double) * (size_t)partial_doubles);
    const size_t need = need_counter + need_split + need_partial;
    OTOO_REQUIRE(need <= kStaticScratchBytes, OTOO_EINVAL,
                 "otoo_force_static: this step needs %zu bytes of scratch, the library array holds %zu "
                 "(32 bytes per source for OTOO_FP32K plus 8 per partial double); use otoo_force",
                 need, kStaticScratchBytes);
    void* base = nullptr;
    int rc = static_scratch_ptr(&base);
    if (rc) return rc;
    otoo_dev_system s = *sys;
    unsigned char* b = static_cast<unsigned char*>(base);
    s.counter = reinterpret_cast<uint32_t*>(b);
    s.split = need_split ? b + need_counter : nullptr;
    s.partial = need_partial ? reinterpret_cast<double*>(b + need_counter + need_split) : nullptr;
    s.partial_doubles = partial_doubles;
    rc = validate_sys(&s);
    if (rc) return rc;
    rc = check_tune(tune);
    if (rc) return rc;
    return enqueue_force(&s, accel, pot, precision, tune, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int otoo_force_static_status(void* stream)
{
    void* base = nullptr;
    int rc = static_scratch_ptr(&base);
    if (rc) return rc;
    return read_status(static_cast<const uint32_t*>(base), stream);
}
