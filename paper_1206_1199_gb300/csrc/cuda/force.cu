// Device half of the force step: every particle of a group against every
// entry of the group's shared interaction list.
//
// Paper: Section II (particle-particle and particle-cell interactions, the
// cell acting as a virtual particle at its centre of mass), Section III-C
// (the GPU evaluates the interactions of a group that shares one walk).  The
// quadrupole cell term, the FP32 centre-relative arithmetic with per-thread
// Kahan sums, the persistent load-balanced launch and the CUDA graph are this
// library's design for sm_103a; the pair law with Plummer softening is a
// reading (the paper keeps a softening length per particle but does not print
// the law).
//
// Kernels
//   k_force<float>   FP32 pairs on group-centre-relative coordinates (the
//                    centre subtraction is FP64, once per staged entry),
//                    plain FP32 sums over a tile, Kahan-compensated across
//                    tiles, FP64 merge of the thread-level j-split and output.
//   k_force<double>  every pair in FP64 (the comparison form).
//   k_merge          FP64 sum of the chunk partials of split lists, in chunk
//                    order (deterministic), plus the self-pair correction.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../common.h"

using namespace otoo;

namespace {

template <typename R> struct V4;
template <> struct __align__(16) V4<float> { float x, y, z, w; };
template <> struct __align__(32) V4<double> { double x, y, z, w; };
template <typename R> struct V2;
template <> struct __align__(8) V2<float> { float x, y; };
template <> struct __align__(16) V2<double> { double x, y; };

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// Status bits written to counter[1].
constexpr uint32_t kBadItem = 1u;
constexpr uint32_t kBadIndex = 2u;

// Accumulator of one target particle: tile partial p, running sum s and
// Kahan compensation c (FP32); FP64 keeps the running sum only.
template <typename R> struct Acc {
    R s[4], c[4];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int k = 0; k < 4; ++k) s[k] = c[k] = R(0);
    }
    __device__ __forceinline__ void add(const R p[4]);
    __device__ __forceinline__ double value(int k) const;
};
template <> __device__ __forceinline__ void Acc<float>::add(const float p[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float y = __fsub_rn(p[k], c[k]);
        const float t = __fadd_rn(s[k], y);
        c[k] = __fsub_rn(__fsub_rn(t, s[k]), y);
        s[k] = t;
    }
}
template <> __device__ __forceinline__ double Acc<float>::value(int k) const
{
    return (double)s[k] - (double)c[k];
}
template <> __device__ __forceinline__ void Acc<double>::add(const double p[4])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] += p[k];
}
template <> __device__ __forceinline__ double Acc<double>::value(int k) const { return s[k]; }

// Monopole pair (also a particle entry): r = x_j - x_i,
// a += m r / (r^2 + eps^2)^(3/2), phi -= m / (r^2 + eps^2)^(1/2).
template <typename R>
__device__ __forceinline__ void pair_mono(const V4<R>& s, R xi, R yi, R zi, R eps2, R p[4])
{
    const R rx = s.x - xi, ry = s.y - yi, rz = s.z - zi;
    const R r2 = fma(rx, rx, fma(ry, ry, fma(rz, rz, eps2)));
    const R q = rsqrt_r(r2);
    const R mq = s.w * q;
    const R mq3 = mq * (q * q);
    p[3] -= mq;
    p[0] = fma(mq3, rx, p[0]);
    p[1] = fma(mq3, ry, p[1]);
    p[2] = fma(mq3, rz, p[2]);
}

// Quadrupole cell: with q = (r^2 + eps^2)^(-1/2),
// phi -= m q + (1/2) (r.Q.r) q^5,  a += (m q^3 + (5/2) (r.Q.r) q^7) r - q^5 Q r.
template <typename R>
__device__ __forceinline__ void pair_quad(const V4<R>& s, const V4<R>& qa, const V2<R>& qb, R xi, R yi, R zi,
                                          R eps2, R p[4])
{
    const R rx = s.x - xi, ry = s.y - yi, rz = s.z - zi;
    const R r2 = fma(rx, rx, fma(ry, ry, fma(rz, rz, eps2)));
    const R q = rsqrt_r(r2);
    const R q2 = q * q;
    const R mq = s.w * q;
    const R mq3 = mq * q2;
    // qa = (xx, yy, zz, xy), qb = (xz, yz)
    const R qr0 = fma(qa.x, rx, fma(qa.w, ry, qb.x * rz));
    const R qr1 = fma(qa.w, rx, fma(qa.y, ry, qb.y * rz));
    const R qr2 = fma(qb.x, rx, fma(qb.y, ry, qa.z * rz));
    const R rqr = fma(rx, qr0, fma(ry, qr1, rz * qr2));
    const R q5 = q * (q2 * q2);
    const R t = rqr * q5;
    p[3] -= fma(R(0.5), t, mq);
    const R cr = fma(R(2.5) * t, q2, mq3);
    p[0] = fma(cr, rx, fma(-q5, qr0, p[0]));
    p[1] = fma(cr, ry, fma(-q5, qr1, p[1]));
    p[2] = fma(cr, rz, fma(-q5, qr2, p[2]));
}

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

template <typename R, int B, int IB>
__global__ void __launch_bounds__(B) k_force(const otoo_dev_system sys, double* __restrict__ accel,
                                             double* __restrict__ pot, int T)
{
    extern __shared__ __align__(32) unsigned char smem[];
    V4<R>* s_src = reinterpret_cast<V4<R>*>(smem);
    V4<R>* s_qa = s_src + T;
    V2<R>* s_qb = reinterpret_cast<V2<R>*>(s_qa + T);
    double* s_red = reinterpret_cast<double*>(s_qb + T);
    __shared__ int s_ticket;

    const int tid = threadIdx.x;
    uint32_t* status = sys.counter + 1;

    for (;;) {
        if (tid == 0) s_ticket = (int)atomicAdd(sys.counter, 1u);
        __syncthreads();
        const int it = s_ticket;
        __syncthreads();
        if (it >= sys.n_items) break;

        const otoo_item item = sys.items[it];
        bool ok = item.g >= 0 && item.g < sys.n_groups;
        otoo_group grp;
        if (ok) grp = sys.groups[item.g];
        const int L = ok ? grp.n_cell + grp.n_part : 0;
        ok = ok && grp.count >= 1 && grp.count <= B * IB && grp.first >= 0 &&
             (int64_t)grp.first + grp.count <= sys.n_part && grp.n_cell >= 0 && grp.n_part >= 0 &&
             item.j0 >= 0 && item.j0 <= item.j1 && item.j1 <= L && grp.list_off >= 0 &&
             grp.list_off + L <= sys.n_list && (item.slot < 0 || grp.count <= sys.n_crit_max);
        if (!ok) {
            if (tid == 0) atomicOr(status, kBadItem);
            continue;
        }

        const int ni = grp.count;
        const int P = (ni + IB - 1) / IB;
        const int nsplit = B / P;
        const int islot = tid % P, js = tid / P;
        const bool active = js < nsplit;
        const R eps2 = (R)grp.eps2;
        const double cx = grp.cx, cy = grp.cy, cz = grp.cz;

        R xi[IB], yi[IB], zi[IB];
        Acc<R> acc[IB];
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            const int i = islot + k * P;
            xi[k] = yi[k] = zi[k] = R(0);
            if (active && i < ni) {
                double x, y, z;
                float m;
                load_src(sys.src, (int64_t)grp.first + i, x, y, z, m);
                xi[k] = (R)(x - cx);
                yi[k] = (R)(y - cy);
                zi[k] = (R)(z - cz);
            }
            acc[k].zero();
        }

        const int32_t* lst = sys.list + grp.list_off;
        for (int seg = 0; seg < 2; ++seg) {
            const bool is_cell = seg == 0;
            const int s0 = is_cell ? item.j0 : max(item.j0, grp.n_cell);
            const int s1 = is_cell ? min(item.j1, grp.n_cell) : item.j1;
            const bool quad = is_cell && sys.quad != nullptr;
            for (int base = s0; base < s1; base += T) {
                const int cnt = min(T, s1 - base);
                for (int k = tid; k < cnt; k += B) {
                    const int idx = __ldg(lst + base + k);
                    const bool good = is_cell ? (idx >= sys.n_part && idx < sys.n_src) : (idx >= 0 && idx < sys.n_part);
                    V4<R> v = {R(0), R(0), R(0), R(0)};
                    if (good) {
                        double x, y, z;
                        float m;
                        load_src(sys.src, idx, x, y, z, m);
                        v.x = (R)(x - cx);
                        v.y = (R)(y - cy);
                        v.z = (R)(z - cz);
                        v.w = (R)m;
                    } else {
                        atomicOr(status, kBadIndex);
                    }
                    s_src[k] = v;
                    if (quad) {
                        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
                        if (good) {
                            const float4* qp = reinterpret_cast<const float4*>(sys.quad + (idx - sys.n_part));
                            a = __ldg(qp);
                            b = __ldg(qp + 1);
                        }
                        s_qa[k] = V4<R>{(R)a.x, (R)a.y, (R)a.z, (R)a.w};
                        s_qb[k] = V2<R>{(R)b.x, (R)b.y};
                    }
                }
                __syncthreads();
                if (active) {
                    R p[IB][4];
#pragma unroll
                    for (int k = 0; k < IB; ++k) p[k][0] = p[k][1] = p[k][2] = p[k][3] = R(0);
                    if (quad) {
#pragma unroll 2
                        for (int j = js; j < cnt; j += nsplit) {
                            const V4<R> s = s_src[j];
                            const V4<R> qa = s_qa[j];
                            const V2<R> qb = s_qb[j];
#pragma unroll
                            for (int k = 0; k < IB; ++k) pair_quad(s, qa, qb, xi[k], yi[k], zi[k], eps2, p[k]);
                        }
                    } else {
#pragma unroll 4
                        for (int j = js; j < cnt; j += nsplit) {
                            const V4<R> s = s_src[j];
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

        // merge the thread-level j-split in FP64, in split order
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
            if (item.slot < 0) {
                const int64_t t = (int64_t)grp.first + i;
                const int64_t o = sys.perm ? sys.perm[t] : t;
                double x, y, z;
                float m;
                load_src(sys.src, t, x, y, z, m);
                // the self pair (r = 0) added -m_i / eps; take it out
                a[3] += (double)m / sqrt(grp.eps2);
                accel[3 * o] = a[0];
                accel[3 * o + 1] = a[1];
                accel[3 * o + 2] = a[2];
                pot[o] = a[3];
            } else {
                double* dst = sys.partial + ((int64_t)item.slot * sys.n_crit_max + i) * 4;
#pragma unroll
                for (int c = 0; c < 4; ++c) dst[c] = a[c];
            }
        }
        __syncthreads();
    }
}

// Sum the chunk partials of each split list in chunk order.
__global__ void k_merge(const otoo_dev_system sys, double* __restrict__ accel, double* __restrict__ pot)
{
    const otoo_split sp = sys.splits[blockIdx.x];
    if (sp.g < 0 || sp.g >= sys.n_groups) {
        if (threadIdx.x == 0) atomicOr(sys.counter + 1, kBadItem);
        return;
    }
    const otoo_group grp = sys.groups[sp.g];
    if (grp.count > sys.n_crit_max || grp.first < 0 || (int64_t)grp.first + grp.count > sys.n_part) {
        if (threadIdx.x == 0) atomicOr(sys.counter + 1, kBadItem);
        return;
    }
    for (int i = threadIdx.x; i < grp.count; i += blockDim.x) {
        double a[4] = {0, 0, 0, 0};
        for (int c = 0; c < sp.n_chunks; ++c) {
            const double* s = sys.partial + ((int64_t)(sp.slot0 + c) * sys.n_crit_max + i) * 4;
#pragma unroll
            for (int k = 0; k < 4; ++k) a[k] += s[k];
        }
        const int64_t t = (int64_t)grp.first + i;
        const int64_t o = sys.perm ? sys.perm[t] : t;
        double x, y, z;
        float m;
        load_src(sys.src, t, x, y, z, m);
        a[3] += (double)m / sqrt(grp.eps2);
        accel[3 * o] = a[0];
        accel[3 * o + 1] = a[1];
        accel[3 * o + 2] = a[2];
        pot[o] = a[3];
    }
}

// ---------------------------------------------------------------------------
// host side: launch configuration, CUDA graph cache

template <typename R>
size_t smem_bytes(int B, int IB, int T)
{
    return (size_t)T * (2 * sizeof(V4<R>) + sizeof(V2<R>)) + (size_t)B * IB * 4 * sizeof(double);
}

using KernelFn = void (*)(const otoo_dev_system, double*, double*, int);

template <typename R>
KernelFn pick_kernel(int B, int IB)
{
    if (B == 128 && IB == 1) return k_force<R, 128, 1>;
    if (B == 128 && IB == 2) return k_force<R, 128, 2>;
    if (B == 256 && IB == 1) return k_force<R, 256, 1>;
    if (B == 256 && IB == 2) return k_force<R, 256, 2>;
    if (B == 256 && IB == 4) return k_force<R, 256, 4>;
    return nullptr;
}

int check_tune(const otoo_tune* t, int n_crit_max)
{
    OTOO_REQUIRE(t, OTOO_EINVAL, "tune is NULL");
    OTOO_REQUIRE(t->tile >= 16 && t->tile <= 1024, OTOO_EINVAL, "tile %d out of [16, 1024]", t->tile);
    OTOO_REQUIRE(pick_kernel<float>(t->block, t->iblock) != nullptr, OTOO_EINVAL,
                 "unsupported block %d / iblock %d", t->block, t->iblock);
    OTOO_REQUIRE(t->block * t->iblock >= n_crit_max, OTOO_EINVAL, "block*iblock = %d < largest group %d",
                 t->block * t->iblock, n_crit_max);
    OTOO_REQUIRE(t->ctas_per_sm >= 0 && t->ctas_per_sm <= 32, OTOO_EINVAL, "ctas_per_sm out of range");
    return OTOO_OK;
}

#define CUDA_TRY(expr)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return set_error(OTOO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

// Records the launches of one force step on stream s.
int enqueue_force(const otoo_dev_system* sys, double* accel, double* pot, int precision, const otoo_tune* t,
                  cudaStream_t s)
{
    const bool fp64 = precision == OTOO_FP64;
    KernelFn fn = fp64 ? pick_kernel<double>(t->block, t->iblock) : pick_kernel<float>(t->block, t->iblock);
    const size_t sm = fp64 ? smem_bytes<double>(t->block, t->iblock, t->tile)
                           : smem_bytes<float>(t->block, t->iblock, t->tile);
    CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int dev = 0, nsm = 0, occ = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t->block, sm));
    if (occ < 1) return set_error(OTOO_EINVAL, "force kernel does not fit on an SM (smem %zu)", sm);
    const int per_sm = t->ctas_per_sm > 0 ? std::min(t->ctas_per_sm, occ) : occ;
    const int grid = (int)std::min<int64_t>(sys->n_items, (int64_t)nsm * per_sm);
    CUDA_TRY(cudaMemsetAsync(sys->counter, 0, 2 * sizeof(uint32_t), s));
    if (grid > 0) {
        fn<<<grid, t->block, sm, s>>>(*sys, accel, pot, t->tile);
        CUDA_TRY(cudaGetLastError());
    }
    if (sys->n_splits > 0) {
        k_merge<<<sys->n_splits, 128, 0, s>>>(*sys, accel, pot);
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
    OTOO_REQUIRE(sys->n_groups >= 1 && sys->n_items >= 1 && sys->n_splits >= 0 && sys->n_list >= 1, OTOO_EINVAL,
                 "bad counts");
    OTOO_REQUIRE(sys->n_crit_max >= 1 && sys->n_crit_max <= kMaxGroup, OTOO_EINVAL, "n_crit_max out of range");
    OTOO_REQUIRE(sys->src && sys->groups && sys->list && sys->items && sys->counter, OTOO_EINVAL,
                 "NULL device array");
    OTOO_REQUIRE(sys->n_splits == 0 || (sys->splits && sys->partial), OTOO_EINVAL, "split lists need partial scratch");
    return OTOO_OK;
}

}  // namespace

extern "C" {

int otoo_force(const otoo_dev_system* sys, double* accel, double* pot, int32_t precision, const otoo_tune* tune,
               void* stream)
{
    int rc = validate_sys(sys);
    if (rc) return rc;
    OTOO_REQUIRE(accel && pot, OTOO_EINVAL, "accel/pot is NULL");
    OTOO_REQUIRE(precision == OTOO_FP32K || precision == OTOO_FP64, OTOO_EINVAL, "bad precision %d", precision);
    rc = check_tune(tune, sys->n_crit_max);
    if (rc) return rc;
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
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t h[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(h, sys->counter, sizeof(h), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (h[1] & kBadItem) return set_error(OTOO_EDEVICE, "a work item or group failed its bounds check");
    if (h[1] & kBadIndex) return set_error(OTOO_EDEVICE, "a list entry indexed outside its source range");
    return OTOO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// otoo_force_host: host arrays in, host arrays out (device buffers cached)

namespace {

struct HostPathBuffers {
    int device = -1;
    void* p[9] = {nullptr};
    size_t cap[9] = {0};
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

extern "C" int otoo_force_host(const otoo_lists_view* lv, const otoo_plan_info* pl, double* accel, double* pot,
                               int32_t precision, const otoo_tune* tune, void* stream)
{
    OTOO_REQUIRE(lv && pl && accel && pot, OTOO_EINVAL, "otoo_force_host: NULL argument");
    OTOO_REQUIRE(lv->n_part >= 1 && lv->n_groups >= 1 && lv->n_list >= 1 && pl->n_items >= 1, OTOO_EINVAL,
                 "otoo_force_host: empty input");
    std::lock_guard<std::mutex> lock(g_host_mu);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (g_host.device != dev) {
        for (int k = 0; k < 9; ++k) g_host.p[k] = nullptr, g_host.cap[k] = 0;  // buffers of another device stay
        g_host.device = dev;
    }
    const int64_t nc = lv->n_src - lv->n_part;
    const size_t bytes[9] = {sizeof(otoo_src) * (size_t)lv->n_src,
                             sizeof(otoo_quad) * (size_t)std::max<int64_t>(nc, 1),
                             sizeof(otoo_group) * (size_t)lv->n_groups,
                             sizeof(int32_t) * (size_t)lv->n_list,
                             sizeof(otoo_item) * (size_t)pl->n_items,
                             sizeof(otoo_split) * (size_t)std::max<int64_t>(pl->n_splits, 1),
                             sizeof(int64_t) * (size_t)lv->n_part,
                             sizeof(double) * (size_t)(std::max<int64_t>(pl->partial_doubles, 1) + 4 * lv->n_part),
                             sizeof(uint32_t) * 4};
    for (int k = 0; k < 9; ++k) {
        int rc = ensure(k, bytes[k]);
        if (rc) return rc;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemcpyAsync(g_host.p[0], lv->src, bytes[0], cudaMemcpyHostToDevice, s));
    if (lv->use_quad && nc > 0) CUDA_TRY(cudaMemcpyAsync(g_host.p[1], lv->quad, bytes[1], cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(g_host.p[2], lv->groups, bytes[2], cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(g_host.p[3], lv->list, bytes[3], cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(g_host.p[4], pl->items, bytes[4], cudaMemcpyHostToDevice, s));
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
    sys.counter = (uint32_t*)g_host.p[8];
    int rc = otoo_force(&sys, out, out + 3 * lv->n_part, precision, tune, stream);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpyAsync(accel, out, sizeof(double) * 3 * (size_t)lv->n_part, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(pot, out + 3 * lv->n_part, sizeof(double) * (size_t)lv->n_part, cudaMemcpyDeviceToHost, s));
    return otoo_check_status(&sys, stream);
}
