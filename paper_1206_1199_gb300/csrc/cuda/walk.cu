// The tree walk on the device and the device work plan.
//
// Paper: Section III-D (the walk runs on the GPU; a group of particles
// shares one traversal and the acceptance test uses the group-to-cell
// minimum distance, after Barnes 1990) and Section II-A (the traversal rules:
// accept a cell, open a cell into its children, take a leaf's particles).
// The paper walks with one work-item per group along next/more links; here
// one warp walks one group over a shared-memory stack, 32 cells at a time,
// and writes the group's list for the force kernels (the host walk's lists,
// entry for entry, as sets per group).
//
// Kernels
//   k_walk<false>   pass 1: the group's box (warp min/max over its particles),
//                   the walk, entry counts into the group record.
//   k_scan_*        exclusive prefix sums in group order (list offsets, plan
//                   slots): block sums, one-CTA scan of the block sums,
//                   block-level scans with the block offsets.
//   k_walk<true>    pass 2: the same walk, entries written at the offsets.
//   k_plan_count    per group: particle and list chunks (the cost model of the
//                   host plan), cost class histogram.
//   k_plan_cursor   start of each cost class, most expensive class first.
//   k_plan_fill     work items and split records.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../common.h"
#include "../plan_chunks.h"

using namespace otoo;

namespace {

constexpr int kWalkWarps = 8;       // warps per CTA
#ifndef OTOO_WALK_HALVES
#define OTOO_WALK_HALVES 2
#endif
constexpr int kWalkHalves = OTOO_WALK_HALVES;  // cells per lane per walk step
#ifndef OTOO_WALK_MIN_BLOCKS
#define OTOO_WALK_MIN_BLOCKS 3  // resident CTAs per SM asked of the register allocator (85 registers)
#endif
constexpr int kWide = 32 * kWalkHalves;         // cells per walk step at most
constexpr int kStack = 512;         // stack entries (runs of sibling cells) per warp
constexpr int kMaxLevels = 22;      // tree levels (root level 0 to the 2^21 grid level)
constexpr int kScanThreads = 1024;  // scan kernels: threads per CTA
constexpr int kScanBlock = 2048;    // elements per scan block
constexpr int kClasses = 128;       // cost classes of the plan's launch order
constexpr int kTotals = 6;          // walk totals: entries, interactions, cell interactions,
                                    // largest n_cell, largest n_part, groups beyond their slots

#include "pair.cuh"

// status bits (counter[1])
constexpr uint32_t kWalkBadRecord = 1u;   // a cell record failed its bounds check
constexpr uint32_t kWalkOverflow = 2u;    // a group's stack or node budget ran out
constexpr uint32_t kWalkMismatch = 4u;    // pass 2 counted other entries than pass 1
constexpr uint32_t kWalkNoRoom = 8u;      // the output array is too small
constexpr uint32_t kWalkBadGroup = 16u;   // a group range failed its check

struct WalkArgs {
    int64_t n_part, n_cell;
    int32_t n_groups, exact, mac, pad;
    double theta, eps2;
    const otoo_src* src;
    const otoo_wcell* cell;
    const otoo_wcell64* cell64;
    const int32_t* gfirst;
    const int32_t* gcount;
    const float* tpg;
    uint32_t* counter;
    int64_t* totals;
};

// Per-group FP32 data of the filter: the group centre c as a float pair and
// the box relative to c.
struct BoxF {
    float c32[3], cl32[3], bl[3], bh[3];
    float B;    // sum over axes of max(|bl|, |bh|)
    float A;    // sum of |c32|: scale of the float-pair truncation error
};

// The acceptance test of the host walk, operation for operation in FP64
// (no contraction: every operation is an explicitly rounded intrinsic).
// Called for the few tests the FP32 filter cannot decide, so kept out of line
// (a smaller walk loop for the instruction cache).
__device__ __noinline__ bool mac_exact(const otoo_wcell64* __restrict__ c64, int k, const double blo[3],
                                       const double bhi[3], double theta)
{
    if (!(theta > 0.0)) return false;
    const otoo_wcell64 c = c64[k];
    bool overlap = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double chi = __dadd_rn(c.lo[a], c.side);
        if (!(c.lo[a] <= bhi[a] && blo[a] <= chi)) overlap = false;
    }
    if (overlap) return false;
    double d2 = 0.0, s2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double d = 0.0;
        const double t0 = __dsub_rn(blo[a], c.com[a]);
        if (t0 > d) d = t0;
        const double t1 = __dsub_rn(c.com[a], bhi[a]);
        if (t1 > d) d = t1;
        d2 = __dadd_rn(d2, __dmul_rn(d, d));
        const double e = __dsub_rn(c.com[a], c.gc[a]);
        s2 = __dadd_rn(s2, __dmul_rn(e, e));
    }
    return __dsqrt_rn(d2) > __dadd_rn(__ddiv_rn(c.side, theta), __dsqrt_rn(s2));
}

// FP32 filter of the acceptance test: 1 = accept, 0 = reject, -1 = too close
// to call.  Without kOverlap (opening angles below 1/sqrt(3)) the cube
// overlap part is left out: a cube that overlaps the box puts its centre of
// mass within sqrt(3) l of the box, below l / theta + s, so the distance part
// alone already rejects it.  u = com - c from the float pairs; every rounded quantity is
// within 2^-20 K of its exact value (K: sum of the magnitudes the test
// combines, plus 2^-24 of the absolute coordinates for the truncated low
// words), so a comparison decided by more than 2^-18 K (box overlap) or
// 2^-16 K^2 (squared distances) is decided the same way by the exact
// arithmetic and by the host's FP64.
template <bool kOverlap>
__device__ __forceinline__ int mac_filter(const otoo_wcell& w, const BoxF& g, float invth)
{
    float u[3], au = 0.f, A = g.A;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = __fadd_rn(__fsub_rn(w.com_hi[a], g.c32[a]), __fsub_rn(w.com_lo[a], g.cl32[a]));
        au += fabsf(u[a]);
        A += fabsf(w.com_hi[a]);
    }
    const float thr = __fadd_rn(__fmul_rn(w.side, invth), w.s);
    const float K = au + g.B + thr + w.side + A * 0x1p-24f;
    if (kOverlap) {
        const float del = K * 0x1p-18f;
        bool sep = false, ovl = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float lo = __fsub_rn(u[a], w.e[a]);
            const float hi = __fadd_rn(lo, w.side);
            sep = sep || (lo > g.bh[a] + del) || (g.bl[a] > hi + del);
            ovl = ovl && (lo < g.bh[a] - del) && (g.bl[a] < hi - del);
        }
        if (ovl) return 0;
        if (!sep) return -1;
    }
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = fmaxf(0.f, fmaxf(g.bl[a] - u[a], u[a] - g.bh[a]));
        d2 = fmaf(d, d, d2);
    }
    const float thr2 = thr * thr, m = K * K * 0x1p-16f;
    if (d2 > thr2 + m) return 1;
    if (d2 < thr2 - m) return 0;
    return -1;
}

// One 32-byte sector per load (256-bit vector loads, sm_100 and later): the
// 64-byte record in two requests instead of four.
__device__ __forceinline__ void ld256(const void* p, float v[8])
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}

// The absolute MAC of the host walk (Eq. SW_MAC): d_min > r_b, FP64,
// operation for operation (out of line, as mac_exact).
__device__ __noinline__ bool sw_exact(const otoo_wcell64* __restrict__ c64, int k, const double blo[3],
                                      const double bhi[3])
{
    const otoo_wcell64 c = c64[k];
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double d = 0.0;
        const double t0 = __dsub_rn(blo[a], c.com[a]);
        if (t0 > d) d = t0;
        const double t1 = __dsub_rn(c.com[a], bhi[a]);
        if (t1 > d) d = t1;
        d2 = __dadd_rn(d2, __dmul_rn(d, d));
    }
    return __dsqrt_rn(d2) > c.rb;
}

// FP32 filter of the absolute MAC with the same bound as mac_filter: the
// squared distance against r_b^2 decides when they differ by more than
// 2^-16 K^2 (K now includes r_b, rounded once from the host's FP64 value).
__device__ __forceinline__ int mac_filter_sw(const otoo_wcell& w, const BoxF& g)
{
    const float rb = w.rb;
    if (!(rb <= 3.0e38f)) return 0;  // infinite r_b (delta = 0): nothing is accepted
    float u[3], au = 0.f, A = g.A;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = __fadd_rn(__fsub_rn(w.com_hi[a], g.c32[a]), __fsub_rn(w.com_lo[a], g.cl32[a]));
        au += fabsf(u[a]);
        A += fabsf(w.com_hi[a]);
    }
    const float K = au + g.B + rb + A * 0x1p-24f;
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = fmaxf(0.f, fmaxf(g.bl[a] - u[a], u[a] - g.bh[a]));
        d2 = fmaf(d, d, d2);
    }
    const float rb2 = rb * rb, m = K * K * 0x1p-16f;
    if (d2 > rb2 + m) return 1;
    if (d2 < rb2 - m) return 0;
    return -1;
}

// mac_filter and mac_filter_sw with the parts that depend on the cell alone
// computed once per cell by the caller (the set walk tests one cell against
// several groups): acell = |com_hi[0]| + |com_hi[1]| + |com_hi[2]| and, for
// the opening angle, thr = side / theta + s as mac_filter rounds it.  Only K
// (the scale of the rounding bound) is summed in another order, which moves
// it by a few FP32 roundings, far inside the margins.
template <bool kOverlap>
__device__ __forceinline__ int mac_filter_pc(const otoo_wcell& w, const BoxF& g, float acell, float thr)
{
    float u[3], au = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = __fadd_rn(__fsub_rn(w.com_hi[a], g.c32[a]), __fsub_rn(w.com_lo[a], g.cl32[a]));
        au += fabsf(u[a]);
    }
    const float K = au + g.B + thr + w.side + (g.A + acell) * 0x1p-24f;
    if (kOverlap) {
        const float del = K * 0x1p-18f;
        bool sep = false, ovl = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float lo = __fsub_rn(u[a], w.e[a]);
            const float hi = __fadd_rn(lo, w.side);
            sep = sep || (lo > g.bh[a] + del) || (g.bl[a] > hi + del);
            ovl = ovl && (lo < g.bh[a] - del) && (g.bl[a] < hi - del);
        }
        if (ovl) return 0;
        if (!sep) return -1;
    }
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = fmaxf(0.f, fmaxf(g.bl[a] - u[a], u[a] - g.bh[a]));
        d2 = fmaf(d, d, d2);
    }
    const float thr2 = thr * thr, m = K * K * 0x1p-16f;
    if (d2 > thr2 + m) return 1;
    if (d2 < thr2 - m) return 0;
    return -1;
}

__device__ __forceinline__ int mac_filter_sw_pc(const otoo_wcell& w, const BoxF& g, float acell)
{
    const float rb = w.rb;
    if (!(rb <= 3.0e38f)) return 0;
    float u[3], au = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = __fadd_rn(__fsub_rn(w.com_hi[a], g.c32[a]), __fsub_rn(w.com_lo[a], g.cl32[a]));
        au += fabsf(u[a]);
    }
    const float K = au + g.B + rb + (g.A + acell) * 0x1p-24f;
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = fmaxf(0.f, fmaxf(g.bl[a] - u[a], u[a] - g.bh[a]));
        d2 = fmaf(d, d, d2);
    }
    const float rb2 = rb * rb, m = K * K * 0x1p-16f;
    if (d2 > rb2 + m) return 1;
    if (d2 < rb2 - m) return 0;
    return -1;
}

__device__ __forceinline__ otoo_wcell load_wcell(const otoo_wcell* __restrict__ cell, int k)
{
    float v[16];
    ld256(cell + k, v);
    ld256(reinterpret_cast<const char*>(cell + k) + 32, v + 8);
    otoo_wcell w;
    w.com_hi[0] = v[0], w.com_hi[1] = v[1], w.com_hi[2] = v[2];
    w.com_lo[0] = v[3], w.com_lo[1] = v[4], w.com_lo[2] = v[5];
    w.e[0] = v[6], w.e[1] = v[7], w.e[2] = v[8];
    w.side = v[9];
    w.s = v[10];
    w.child0 = __float_as_int(v[11]);
    w.nchild = __float_as_int(v[12]);
    w.begin = __float_as_int(v[13]);
    w.end = __float_as_int(v[14]);
    w.rb = v[15];
    return w;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Order-preserving integer key of a double (for non-NaN values): min/max on
// the keys is min/max on the values, on the integer pipe.
__device__ __forceinline__ long long dkey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dval(long long k) { return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL)); }

__device__ __forceinline__ long long warp_min(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(kFull, v, o);
        v = t < v ? t : v;
    }
    return v;
}
__device__ __forceinline__ long long warp_max(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long t = __shfl_xor_sync(kFull, v, o);
        v = t > v ? t : v;
    }
    return v;
}

// A stack entry is a run of consecutive cells (the children of one cell):
// first cell in the low 28 bits, run length - 1 (0..7) above.
constexpr uint32_t kRunShift = 28;
constexpr uint32_t kRunMask = (1u << kRunShift) - 1u;
__device__ __forceinline__ uint32_t run(int first, int n) { return (uint32_t)first | ((uint32_t)(n - 1) << kRunShift); }

// Geometry and acceptance rule of one group's walk.
struct GroupWalk {
    double blo[3], bhi[3], c[3];  // the particles' box (exact) and its centre
    BoxF bf;
    double theta;                 // opening angle of this group (0 for the absolute MAC / SPH)
    float invth;                  // 1 / theta rounded to FP32
    bool sw;                      // absolute MAC or SPH radius: accept when d_min > r_b
    bool drop;                    // SPH: accepted cells enter no list
    bool open_all;                // opening angle 0: nothing is accepted
    bool small_angle;             // theta < 1/sqrt(3): the filter skips the cube-overlap part
};

// The box of particles [first, first + count) (min/max on order-preserving
// integer keys, exact), its FP32 form for the filter, and the group's rule.
__device__ __forceinline__ void group_walk_setup(const WalkArgs& a, int g, int32_t first, int32_t count, int lane,
                                                 GroupWalk& w)
{
    long long klo[3], khi[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) klo[k] = 0x7fffffffffffffffLL, khi[k] = -klo[k] - 1;
    for (int i = lane; i < count; i += 32) {
        const double2* ps = reinterpret_cast<const double2*>(a.src + first + i);
        const double2 xy = __ldg(ps), zm = __ldg(ps + 1);
        const long long kx = dkey(xy.x), ky = dkey(xy.y), kz = dkey(zm.x);
        klo[0] = kx < klo[0] ? kx : klo[0], khi[0] = kx > khi[0] ? kx : khi[0];
        klo[1] = ky < klo[1] ? ky : klo[1], khi[1] = ky > khi[1] ? ky : khi[1];
        klo[2] = kz < klo[2] ? kz : klo[2], khi[2] = kz > khi[2] ? kz : khi[2];
    }
    w.bf.B = 0.f;
    w.bf.A = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        w.blo[k] = dval(warp_min(klo[k]));
        w.bhi[k] = dval(warp_max(khi[k]));
        w.c[k] = __dmul_rn(__dadd_rn(w.blo[k], w.bhi[k]), 0.5);
        w.bf.c32[k] = __double2float_rn(w.c[k]);
        w.bf.cl32[k] = __double2float_rn(__dsub_rn(w.c[k], (double)w.bf.c32[k]));
        w.bf.bl[k] = __double2float_rn(__dsub_rn(w.blo[k], w.c[k]));
        w.bf.bh[k] = __double2float_rn(__dsub_rn(w.bhi[k], w.c[k]));
        w.bf.B += fmaxf(fabsf(w.bf.bl[k]), fabsf(w.bf.bh[k]));
        w.bf.A += fabsf(w.bf.c32[k]);
    }
    // the absolute MAC and the SPH radius share the test d_min > r_b; an
    // SPH walk drops the cells that pass it (no neighbour inside)
    w.sw = a.mac == OTOO_MAC_SW || a.mac == OTOO_MAC_SPH;
    w.drop = a.mac == OTOO_MAC_SPH;
    w.theta = w.sw ? 0.0 : a.tpg ? (double)a.tpg[g] : a.theta;
    // the per-group choices as bits of an integer, taken through an opaque
    // move: the compiler must not re-derive them from theta inside the
    // walk loop, where FP64 compares would occupy GB300's narrow FP64 pipe
    int fl = (!w.sw && !(w.theta > 0.0) ? 1 : 0) | (w.theta < 0.57 ? 2 : 0);  // 0.57 < 1/sqrt(3) = 0.5774
    asm volatile("mov.b32 %0, %0;" : "+r"(fl));
    w.open_all = (fl & 1) != 0;
    w.small_angle = (fl & 2) != 0;
    // 1/theta within 2^-23 (the filter's margins allow 2^-21)
    w.invth = w.open_all ? 0.f : __frcp_rn(__double2float_rn(w.theta));
}

// The cells one walk step took and their decisions: lane j holds positions
// j + 32 h of the taken runs; kind 1 accept, 2 rejected leaf, 3 open, 0 none.
struct StepCells {
    int node[kWalkHalves], kind[kWalkHalves], c0[kWalkHalves], nch[kWalkHalves], pb[kWalkHalves],
        pe[kWalkHalves];
};

// Takes up to kWide cells from the top runs of the stack (the last run may be
// split, its rest goes back) and tests them.  False when the stack or the
// cell budget ran out (the walk stops).
__device__ __forceinline__ bool walk_take(const WalkArgs& a, const GroupWalk& w, uint32_t* stk, int& sp,
                                          int64_t& budget, int lane, StepCells& sc, uint32_t* status)
{
    if (sp + 2 > kStack) return false;
    const int wcap = sp + kWide + 1 + kMaxLevels <= kStack ? kWide : 1;
    // the top runs: lane l reads the l-th entry from the top
    const int nr = sp < 32 ? sp : 32;
    uint32_t e = 0;
    int rn = 0;
    if (lane < nr) {
        e = stk[sp - 1 - lane];
        rn = (int)(e >> kRunShift) + 1;
    }
    const int rinc = warp_incl_scan(rn, lane);
    const int rstart = rinc - rn;
    // runs wholly taken, and a run cut at wcap
    const bool whole = lane < nr && rinc <= wcap;
    const bool cut = lane < nr && rstart < wcap && rinc > wcap;
    const int nwhole = __popc(__ballot_sync(kFull, whole));
    const unsigned cutm = __ballot_sync(kFull, cut);
    const int in_whole = __shfl_sync(kFull, rinc, nwhole > 0 ? nwhole - 1 : 0);
    const int W = cutm ? wcap : (nwhole > 0 ? in_whole : 0);
    // start positions of the taken runs, 32 positions per mask word
    unsigned starts[kWalkHalves];
#pragma unroll
    for (int h = 0; h < kWalkHalves; ++h)
        starts[h] = __reduce_or_sync(kFull, (whole || cut) && rstart >= 32 * h && rstart < 32 * h + 32
                                                ? (1u << (rstart - 32 * h))
                                                : 0u);
    // the run that continues after the cut goes back on the stack first
    sp -= nwhole + (cutm ? 1 : 0);
    if (cut) {
        const int taken = wcap - rstart;
        stk[sp] = run((int)(e & kRunMask) + taken, rn - taken);
    }
    sp += cutm ? 1 : 0;
    budget -= W;
    if (budget < 0) return false;
    // lane j takes the cells at positions j, j + 32, ... of the taken
    // runs; position q lies in the run whose start is the last one <= q
#pragma unroll
    for (int h = 0; h < kWalkHalves; ++h) {
        int r = -1;
#pragma unroll
        for (int k = 0; k <= h; ++k) r += __popc(starts[k] & (k < h ? 0xffffffffu : (2u << lane) - 1u));
        const uint32_t er = __shfl_sync(kFull, e, r < 0 ? 0 : r);
        const int sr = __shfl_sync(kFull, rstart, r < 0 ? 0 : r);
        const int q = lane + 32 * h;
        sc.node[h] = q < W ? (int)(er & kRunMask) + (q - sr) : -1;
        sc.kind[h] = 0;
        sc.c0[h] = sc.nch[h] = sc.pb[h] = sc.pe[h] = 0;
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < kWalkHalves; ++h) {
        if (lane + 32 * h >= W) continue;
        const int nd = sc.node[h];
        bool ok = nd >= 0 && nd < a.n_cell;
        if (ok) {
            const otoo_wcell c = load_wcell(a.cell, nd);
            sc.nch[h] = c.nchild;
            sc.c0[h] = c.child0;
            sc.pb[h] = c.begin;
            sc.pe[h] = c.end;
            ok = sc.nch[h] >= 0 && sc.nch[h] <= 8 &&
                 (sc.nch[h] == 0 || (sc.c0[h] > nd && (int64_t)sc.c0[h] + sc.nch[h] <= a.n_cell)) &&
                 sc.pb[h] >= 0 && sc.pb[h] <= sc.pe[h] && (int64_t)sc.pe[h] <= a.n_part;
            if (ok) {
                int dec = 0;
                if (w.sw) {
                    dec = a.exact ? -1 : mac_filter_sw(c, w.bf);
                    if (dec < 0) dec = sw_exact(a.cell64, nd, w.blo, w.bhi) ? 1 : 0;
                } else if (!w.open_all) {
                    dec = a.exact ? -1
                          : w.small_angle ? mac_filter<false>(c, w.bf, w.invth)
                                          : mac_filter<true>(c, w.bf, w.invth);
                    if (dec < 0) dec = mac_exact(a.cell64, nd, w.blo, w.bhi, w.theta) ? 1 : 0;
                }
                sc.kind[h] = dec ? 1 : (sc.nch[h] == 0 ? 2 : 3);
            }
        }
        if (!ok) atomicOr(status, kWalkBadRecord);
    }
    return true;
}

// One run per rejected inner cell of the step, the lowest position's on top:
// the last positions are pushed first.
__device__ __forceinline__ void walk_push(uint32_t* stk, int& sp, const StepCells& sc, unsigned lt)
{
#pragma unroll
    for (int h = kWalkHalves - 1; h >= 0; --h) {
        const unsigned om = __ballot_sync(kFull, sc.kind[h] == 3);
        const int no = __popc(om);
        if (sc.kind[h] == 3) stk[sp + no - 1 - __popc(om & lt)] = run(sc.c0[h], sc.nch[h]);
        sp += no;
    }
    __syncwarp();
}

// One warp per group (atomic ticket).  The stack holds runs of sibling
// cells; each step takes up to kWide = 32 kWalkHalves cells from the top runs
// (walk_take; lane j tests the cells at positions j, j + 32, ...), emits
// accepted cells and rejected leaves' particles in position order and pushes
// one run per rejected inner cell (its children, walk_push).  A kWide-cell
// step adds at most kWide entries and runs only with kWide + 1 + kMaxLevels
// entries free; otherwise the step takes one cell, which adds at most one
// entry, and only when it descends a level (a tree has at most kMaxLevels
// levels below any cell), so the stack never overflows.
// kMode 0: count (group records, totals); 1: fill the list at the offsets
// of pass 0; 2: single pass -- count as pass 0 and write each group's entries
// into its fixed slot of list (capacity cells + pcap particles per slot):
// cells backwards from slot position capacity - 1, particles forwards from
// capacity, so that they end up contiguous, cells first, and the slots serve
// as the list (list_off set here; groups that outgrow their slot get -1).
template <int kMode>
__global__ void __launch_bounds__(kWalkWarps * 32, OTOO_WALK_MIN_BLOCKS) k_walk(WalkArgs a, otoo_group* __restrict__ groups,
                                                          int32_t* __restrict__ list, int64_t capacity, int64_t pcap)
{
    constexpr bool kFill = kMode == 1;
    constexpr bool kCount = kMode != 1;
    constexpr bool kWrite = kMode != 0;
    __shared__ uint32_t stack_s[kWalkWarps][kStack];
    const int lane = threadIdx.x & 31;
    uint32_t* stk = stack_s[threadIdx.x >> 5];
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* status = a.counter + 1;
    if (kFill && a.totals[0] > capacity) {
        if (threadIdx.x == 0) atomicOr(status, kWalkNoRoom);
        return;
    }
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(a.counter, 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= a.n_groups) break;
        const int32_t first = a.gfirst[g], count = a.gcount[g];
        if (first < 0 || count < 1 || count > kMaxGroup || (int64_t)first + count > a.n_part) {
            if (lane == 0) {
                atomicOr(status, kWalkBadGroup);
                if (kCount) {
                    otoo_group z = {};
                    z.first = first;
                    z.eps2 = a.eps2;
                    z.theta = -1.f;
                    groups[g] = z;
                }
            }
            continue;
        }
        GroupWalk w;
        group_walk_setup(a, g, first, count, lane, w);
        int64_t off_c = 0, off_p = 0;
        int32_t want_c = 0, want_p = 0;
        if (kMode == 2) {
            // cell r at off_c - r, particle k at off_p + k
            off_p = (int64_t)g * (capacity + pcap) + capacity;
            off_c = off_p - 1;
            want_c = (int32_t)capacity;
            want_p = (int32_t)pcap;
        }
        if (kFill) {
            const otoo_group gr = groups[g];
            off_c = gr.list_off;
            want_c = gr.n_cell;
            want_p = gr.n_part;
            off_p = off_c + want_c;
            if (off_c < 0 || want_c < 0 || want_p < 0 || off_p + want_p > capacity) {
                if (lane == 0) atomicOr(status, kWalkNoRoom);
                continue;
            }
        }
        int32_t ncell = 0, npart = 0;
        int sp = 0;
        if (w.theta >= 0.0) {
            if (lane == 0) stk[0] = run(0, 1);
            sp = 1;
        }
        __syncwarp();
        int64_t budget = a.n_cell;  // a tree visits each cell at most once
        bool failed = false;
        while (sp > 0) {
            StepCells sc;
            if (!walk_take(a, w, stk, sp, budget, lane, sc, status)) {
                failed = true;
                break;
            }
            // accepted cells, in position order
#pragma unroll
            for (int h = 0; h < kWalkHalves; ++h) {
                const unsigned am = __ballot_sync(kFull, sc.kind[h] == 1 && !w.drop);
                if (kWrite && sc.kind[h] == 1 && !w.drop) {
                    const int32_t r = ncell + __popc(am & lt);
                    if (r < want_c) list[kMode == 2 ? off_c - r : off_c + r] = (int32_t)(a.n_part + sc.node[h]);
                }
                ncell += __popc(am);
            }
            // particles of rejected leaves, in position order
#pragma unroll
            for (int h = 0; h < kWalkHalves; ++h) {
                if (!__any_sync(kFull, sc.kind[h] == 2)) continue;
                const int np = sc.kind[h] == 2 ? sc.pe[h] - sc.pb[h] : 0;
                const int pin = warp_incl_scan(np, lane);
                if (kWrite && np > 0) {
                    const int32_t base = npart + pin - np;
                    for (int k = 0; k < np; ++k)
                        if (base + k < want_p) list[off_p + base + k] = sc.pb[h] + k;
                }
                npart += __shfl_sync(kFull, pin, 31);
            }
            walk_push(stk, sp, sc, lt);
        }
        if (failed && lane == 0) atomicOr(status, kWalkOverflow);
        if (kCount) {
            if (lane == 0) {
                otoo_group r;
                r.first = first;
                r.count = count;
                r.n_cell = ncell;
                r.n_part = npart;
                // pass 0: the offsets come from the scan that follows
                r.list_off = kMode == 2 ? (ncell <= want_c && npart <= want_p ? off_p - ncell : -1) : 0;
                r.eps2 = a.eps2;
                r.cx = w.c[0];
                r.cy = w.c[1];
                r.cz = w.c[2];
                r.theta = (float)w.theta;
                r.sys = 0;
                groups[g] = r;
                const int64_t len = (int64_t)ncell + npart;
                atomicAdd(reinterpret_cast<unsigned long long*>(a.totals), (unsigned long long)len);
                atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 1), (unsigned long long)(len * count));
                atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 2),
                          (unsigned long long)((int64_t)ncell * count));
                atomicMax(reinterpret_cast<unsigned long long*>(a.totals + 3), (unsigned long long)ncell);
                atomicMax(reinterpret_cast<unsigned long long*>(a.totals + 4), (unsigned long long)npart);
                if (kMode == 2 && (ncell > want_c || npart > want_p))
                    atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 5), 1ull);
            }
        } else if (lane == 0 && (ncell != want_c || npart != want_p)) {
            atomicOr(status, kWalkMismatch);
        }
    }
}


// ---- the walk of a set of groups ----------------------------------------------
//
// Groups that are neighbours in tree order lie close together, and their walks
// test mostly the same cells: for the sets of groups under one parent cell of
// a Hernquist halo (7.6 groups per set at n_crit 128) the per-group walks
// visit 5.9 times as many cells as one walk over the union of their visited
// cells.  k_walk_set walks up to kSet consecutive groups with one warp: every
// stack run carries the mask of the set's groups for which the run's cells
// are still open (all their ancestors rejected), a taken cell's record is
// loaded once and tested against each group of its mask with that group's
// own test (the FP32 filter and the FP64 fallback of k_walk), and each group
// keeps its own counts and list slots.  A cell a group accepts is emitted
// for that group, a rejected leaf's particles go to every group that rejected
// it, and an inner cell rejected by any group is opened with the mask of the
// groups that rejected it.  Restricted to one group, the walk visits exactly
// the cells the group's own walk visits and takes the same decisions, so
// each group's entries are those of k_walk (as sets; the order of a group's
// entries is the union walk's).  The stack bound of k_walk holds unchanged
// (one run per opened cell).

constexpr int kSet = 8;  // groups per set at most (one bit each in a run's mask)

// One group of a set: its rule and box (as GroupWalk) and where its entries go.
struct SetGroup {
    BoxF bf;
    double blo[3], bhi[3], c[3];
    double theta;
    float invth;
    int32_t flags;         // 1: opening angle 0 (nothing accepted), 2: theta < 1/sqrt(3)
    int32_t first, count;
    int64_t off_c, off_p;  // where cell r and particle k go (cells backwards in the single pass)
    int32_t want_c, want_p;
};

// Cells of one set-walk step: lane j holds positions j + 32 h of the taken
// runs; acc / rej: masks of the groups that accept / reject the cell.
struct SetStep {
    int node[kWalkHalves], c0[kWalkHalves], nch[kWalkHalves], pb[kWalkHalves], pe[kWalkHalves];
    unsigned acc[kWalkHalves], rej[kWalkHalves];
};

// The decision of group j of a set on cell nd (record c): 1 accept, 0 reject.
// acell, thr_u: the cell's own parts of the filter (thr_u for the set's
// common angle, used when uni).
__device__ __forceinline__ int set_decide(const WalkArgs& a, const SetGroup& g, bool sw, const otoo_wcell& c, int nd,
                                          float acell, float thr_u, bool uni)
{
    if (sw) {
        int dec = a.exact ? -1 : mac_filter_sw_pc(c, g.bf, acell);
        if (dec < 0) dec = sw_exact(a.cell64, nd, g.blo, g.bhi) ? 1 : 0;
        return dec;
    }
    if (g.flags & 1) return 0;
    const float thr = uni ? thr_u : __fadd_rn(__fmul_rn(c.side, g.invth), c.s);
    int dec = a.exact ? -1 : (g.flags & 2) ? mac_filter_pc<false>(c, g.bf, acell, thr)
                                           : mac_filter_pc<true>(c, g.bf, acell, thr);
    if (dec < 0) dec = mac_exact(a.cell64, nd, g.blo, g.bhi, g.theta) ? 1 : 0;
    return dec;
}

// walk_take for a set: takes up to kWide cells with their runs' masks and
// tests each against the groups of its mask.
__device__ __forceinline__ bool set_take(const WalkArgs& a, const SetGroup* sg, bool sw, float invth_u, bool uni,
                                         uint32_t* stk, uint8_t* msk, int& sp, int64_t& budget, int lane, SetStep& st,
                                         uint32_t* status)
{
    if (sp + 2 > kStack) return false;
    const int wcap = sp + kWide + 1 + kMaxLevels <= kStack ? kWide : 1;
    const int nr = sp < 32 ? sp : 32;
    uint32_t e = 0;
    unsigned em = 0;
    int rn = 0;
    if (lane < nr) {
        e = stk[sp - 1 - lane];
        em = msk[sp - 1 - lane];
        rn = (int)(e >> kRunShift) + 1;
    }
    const int rinc = warp_incl_scan(rn, lane);
    const int rstart = rinc - rn;
    const bool whole = lane < nr && rinc <= wcap;
    const bool cut = lane < nr && rstart < wcap && rinc > wcap;
    const int nwhole = __popc(__ballot_sync(kFull, whole));
    const unsigned cutm = __ballot_sync(kFull, cut);
    const int in_whole = __shfl_sync(kFull, rinc, nwhole > 0 ? nwhole - 1 : 0);
    const int W = cutm ? wcap : (nwhole > 0 ? in_whole : 0);
    unsigned starts[kWalkHalves];
#pragma unroll
    for (int h = 0; h < kWalkHalves; ++h)
        starts[h] = __reduce_or_sync(kFull, (whole || cut) && rstart >= 32 * h && rstart < 32 * h + 32
                                                ? (1u << (rstart - 32 * h))
                                                : 0u);
    sp -= nwhole + (cutm ? 1 : 0);
    if (cut) {
        const int taken = wcap - rstart;
        stk[sp] = run((int)(e & kRunMask) + taken, rn - taken);
        msk[sp] = (uint8_t)em;
    }
    sp += cutm ? 1 : 0;
    budget -= W;
    if (budget < 0) return false;
    unsigned cm[kWalkHalves];
#pragma unroll
    for (int h = 0; h < kWalkHalves; ++h) {
        int r = -1;
#pragma unroll
        for (int k = 0; k <= h; ++k) r += __popc(starts[k] & (k < h ? 0xffffffffu : (2u << lane) - 1u));
        const uint32_t er = __shfl_sync(kFull, e, r < 0 ? 0 : r);
        const int sr = __shfl_sync(kFull, rstart, r < 0 ? 0 : r);
        cm[h] = __shfl_sync(kFull, em, r < 0 ? 0 : r);
        const int q = lane + 32 * h;
        st.node[h] = q < W ? (int)(er & kRunMask) + (q - sr) : -1;
        st.acc[h] = st.rej[h] = 0u;
        st.c0[h] = st.nch[h] = st.pb[h] = st.pe[h] = 0;
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < kWalkHalves; ++h) {
        if (lane + 32 * h >= W) continue;
        const int nd = st.node[h];
        bool ok = nd >= 0 && nd < a.n_cell;
        if (ok) {
            const otoo_wcell c = load_wcell(a.cell, nd);
            st.nch[h] = c.nchild;
            st.c0[h] = c.child0;
            st.pb[h] = c.begin;
            st.pe[h] = c.end;
            ok = st.nch[h] >= 0 && st.nch[h] <= 8 &&
                 (st.nch[h] == 0 || (st.c0[h] > nd && (int64_t)st.c0[h] + st.nch[h] <= a.n_cell)) &&
                 st.pb[h] >= 0 && st.pb[h] <= st.pe[h] && (int64_t)st.pe[h] <= a.n_part;
            if (ok) {
                const float acell = fabsf(c.com_hi[0]) + fabsf(c.com_hi[1]) + fabsf(c.com_hi[2]);
                const float thr_u = __fadd_rn(__fmul_rn(c.side, invth_u), c.s);
                unsigned ac = 0u;
                for (unsigned m = cm[h] & ((1u << kSet) - 1u); m; m &= m - 1u) {
                    const int j = __ffs(m) - 1;
                    if (set_decide(a, sg[j], sw, c, nd, acell, thr_u, uni)) ac |= 1u << j;
                }
                st.acc[h] = ac;
                st.rej[h] = cm[h] & ((1u << kSet) - 1u) & ~ac;
            }
        }
        if (!ok) atomicOr(status, kWalkBadRecord);
    }
    return true;
}

// walk_push for a set: one run per inner cell some group rejected, with the
// mask of the groups that rejected it; the lowest position's run on top.
__device__ __forceinline__ void set_push(uint32_t* stk, uint8_t* msk, int& sp, const SetStep& st, unsigned lt)
{
#pragma unroll
    for (int h = kWalkHalves - 1; h >= 0; --h) {
        const bool op = st.rej[h] != 0u && st.nch[h] > 0;
        const unsigned om = __ballot_sync(kFull, op);
        const int no = __popc(om);
        if (op) {
            const int at = sp + no - 1 - __popc(om & lt);
            stk[at] = run(st.c0[h], st.nch[h]);
            msk[at] = (uint8_t)st.rej[h];
        }
        sp += no;
    }
    __syncwarp();
}

// One warp per set of gs <= kSet consecutive groups (atomic ticket over
// sets); kMode as k_walk's.
template <int kMode>
__global__ void __launch_bounds__(kWalkWarps * 32, OTOO_WALK_MIN_BLOCKS)
    k_walk_set(WalkArgs a, int32_t n_sets, int32_t gs, otoo_group* __restrict__ groups, int32_t* __restrict__ list,
               int64_t capacity, int64_t pcap)
{
    constexpr bool kFill = kMode == 1;
    constexpr bool kCount = kMode != 1;
    constexpr bool kWrite = kMode != 0;
    __shared__ uint32_t stack_s[kWalkWarps][kStack];
    __shared__ uint8_t mask_s[kWalkWarps][kStack];
    __shared__ SetGroup sg_s[kWalkWarps][kSet];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint32_t* stk = stack_s[wid];
    uint8_t* msk = mask_s[wid];
    SetGroup* sg = sg_s[wid];
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* status = a.counter + 1;
    const bool sw = a.mac == OTOO_MAC_SW || a.mac == OTOO_MAC_SPH;
    const bool drop = a.mac == OTOO_MAC_SPH;
    if (kFill && a.totals[0] > capacity) {
        if (threadIdx.x == 0) atomicOr(status, kWalkNoRoom);
        return;
    }
    for (;;) {
        int set = 0;
        if (lane == 0) set = (int)atomicAdd(a.counter, 1u);
        set = __shfl_sync(kFull, set, 0);
        if (set >= n_sets) break;
        const int g0 = set * gs;
        const int ng = min(gs, a.n_groups - g0);
        unsigned live = 0u;   // groups that walk
        unsigned valid = 0u;  // groups with a record to write (pass 0 / single pass) or check (pass 1)
        for (int j = 0; j < ng; ++j) {
            const int g = g0 + j;
            const int32_t first = a.gfirst[g], count = a.gcount[g];
            if (first < 0 || count < 1 || count > kMaxGroup || (int64_t)first + count > a.n_part) {
                if (lane == 0) {
                    atomicOr(status, kWalkBadGroup);
                    if (kCount) {
                        otoo_group z = {};
                        z.first = first;
                        z.eps2 = a.eps2;
                        z.theta = -1.f;
                        groups[g] = z;
                    }
                }
                continue;
            }
            GroupWalk w;
            group_walk_setup(a, g, first, count, lane, w);
            int64_t off_c = 0, off_p = 0;
            int32_t want_c = 0, want_p = 0;
            if (kMode == 2) {
                off_p = (int64_t)g * (capacity + pcap) + capacity;
                off_c = off_p - 1;
                want_c = (int32_t)capacity;
                want_p = (int32_t)pcap;
            }
            if (kFill) {
                const otoo_group gr = groups[g];
                off_c = gr.list_off;
                want_c = gr.n_cell;
                want_p = gr.n_part;
                off_p = off_c + want_c;
                if (off_c < 0 || want_c < 0 || want_p < 0 || off_p + want_p > capacity) {
                    if (lane == 0) atomicOr(status, kWalkNoRoom);
                    continue;
                }
            }
            if (lane == 0) {
                SetGroup& q = sg[j];
                q.bf = w.bf;
#pragma unroll
                for (int k = 0; k < 3; ++k) q.blo[k] = w.blo[k], q.bhi[k] = w.bhi[k], q.c[k] = w.c[k];
                q.theta = w.theta;
                q.invth = w.invth;
                q.flags = (w.open_all ? 1 : 0) | (w.small_angle ? 2 : 0);
                q.first = first;
                q.count = count;
                q.off_c = off_c;
                q.off_p = off_p;
                q.want_c = want_c;
                q.want_p = want_p;
            }
            valid |= 1u << j;
            if (w.theta >= 0.0) live |= 1u << j;
        }
        __syncwarp();
        // one opening angle for all walking groups: the threshold side /
        // theta + s is computed once per cell
        float invth_u = 0.f;
        bool uni = false;
        if (live) {
            invth_u = sg[__ffs(live) - 1].invth;
            uni = true;
            for (unsigned m = live; m; m &= m - 1u) uni = uni && sg[__ffs(m) - 1].invth == invth_u;
        }
        int my_nc = 0, my_np = 0;  // lane j: counts of group j
        int sp = 0;
        if (live) {
            if (lane == 0) {
                stk[0] = run(0, 1);
                msk[0] = (uint8_t)live;
            }
            sp = 1;
        }
        __syncwarp();
        int64_t budget = a.n_cell;  // the union of the walks visits each cell at most once
        bool failed = false;
        while (sp > 0) {
            SetStep st;
            if (!set_take(a, sg, sw, invth_u, uni, stk, msk, sp, budget, lane, st, status)) {
                failed = true;
                break;
            }
            // accepted cells, per group, in position order
            unsigned acc_any = 0u, leaf_any = 0u;
#pragma unroll
            for (int h = 0; h < kWalkHalves; ++h) {
                acc_any |= st.acc[h];
                leaf_any |= st.nch[h] == 0 ? st.rej[h] : 0u;
            }
            acc_any = drop ? 0u : __reduce_or_sync(kFull, acc_any);
            leaf_any = __reduce_or_sync(kFull, leaf_any);
            // (loops over the groups present, not unrolled: the walk loop must
            // stay small for the instruction cache)
#pragma unroll 1
            for (unsigned gm = acc_any; gm; gm &= gm - 1u) {
                const int j = __ffs(gm) - 1;
                const int64_t oc = sg[j].off_c;
                const int32_t wc = sg[j].want_c;
                int n = __shfl_sync(kFull, my_nc, j);
#pragma unroll
                for (int h = 0; h < kWalkHalves; ++h) {
                    const bool mine = (st.acc[h] >> j) & 1u;
                    const unsigned am = __ballot_sync(kFull, mine);
                    if (kWrite && mine) {
                        const int32_t r = n + __popc(am & lt);
                        if (r < wc) list[kMode == 2 ? oc - r : oc + r] = (int32_t)(a.n_part + st.node[h]);
                    }
                    n += __popc(am);
                }
                if (lane == j) my_nc = n;
            }
            // particles of rejected leaves, per group, in position order
#pragma unroll 1
            for (unsigned gm = leaf_any; gm; gm &= gm - 1u) {
                const int j = __ffs(gm) - 1;
                const int64_t op = sg[j].off_p;
                const int32_t wp = sg[j].want_p;
                int n = __shfl_sync(kFull, my_np, j);
#pragma unroll
                for (int h = 0; h < kWalkHalves; ++h) {
                    const bool mine = st.nch[h] == 0 && ((st.rej[h] >> j) & 1u);
                    if (!__any_sync(kFull, mine)) continue;
                    const int np = mine ? st.pe[h] - st.pb[h] : 0;
                    const int pin = warp_incl_scan(np, lane);
                    if (kWrite && np > 0) {
                        const int32_t base = n + pin - np;
                        for (int k = 0; k < np; ++k)
                            if (base + k < wp) list[op + base + k] = st.pb[h] + k;
                    }
                    n += __shfl_sync(kFull, pin, 31);
                }
                if (lane == j) my_np = n;
            }
            set_push(stk, msk, sp, st, lt);
        }
        if (failed && lane == 0) atomicOr(status, kWalkOverflow);
        // the groups' records (lane j writes group j's)
        const int nc = my_nc, npt = my_np;
        const bool mine = lane < ng && ((valid >> lane) & 1u);
        if (mine) {
            const SetGroup& q = sg[lane];
            if (kCount) {
                otoo_group r;
                r.first = q.first;
                r.count = q.count;
                r.n_cell = nc;
                r.n_part = npt;
                r.list_off = kMode == 2 ? (nc <= q.want_c && npt <= q.want_p ? q.off_p - nc : -1) : 0;
                r.eps2 = a.eps2;
                r.cx = q.c[0];
                r.cy = q.c[1];
                r.cz = q.c[2];
                r.theta = (float)q.theta;
                r.sys = 0;
                groups[g0 + lane] = r;
                const int64_t len = (int64_t)nc + npt;
                atomicAdd(reinterpret_cast<unsigned long long*>(a.totals), (unsigned long long)len);
                atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 1), (unsigned long long)(len * q.count));
                atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 2),
                          (unsigned long long)((int64_t)nc * q.count));
                atomicMax(reinterpret_cast<unsigned long long*>(a.totals + 3), (unsigned long long)nc);
                atomicMax(reinterpret_cast<unsigned long long*>(a.totals + 4), (unsigned long long)npt);
                if (kMode == 2 && (nc > q.want_c || npt > q.want_p))
                    atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 5), 1ull);
            } else if (nc != q.want_c || npt != q.want_p) {
                atomicOr(status, kWalkMismatch);
            }
        }
        __syncwarp();
    }
}

// ---- the walk fused with the force (the paper's GPU design) ------------------
// One warp per group walks the tree as k_walk does, but the entries do not go
// to a list in device memory: accepted cells and the particles of rejected
// leaves collect in two shared-memory index buffers, and whenever one holds a
// tile of entries the warp stages the tile as pair records (the layout of
// k_force_warp2) and evaluates it against the group's particles, IB per lane
// in lane subsets, with packed FP32 pairs and per-tile Kahan sums.  No list,
// no plan, no work items: the group is the work item.
constexpr int kFuseWarps = 4;                 // warps per CTA
constexpr int kFuseTP = 128;                  // pair records per tile at most
constexpr int kFusePPL = kFuseTP / 32;        // pair records staged per lane
constexpr int kFuseBuf = 2 * kFuseTP + kWide; // index buffer: a tile plus one step's cells

struct FuseArgs {
    const float4* split;    // [2 n_src] float pairs of the sources
    const otoo_quad* quad;  // [n_cell] or NULL (monopole cells)
    const int64_t* perm;    // [n_part] tree order -> caller order, or NULL
    double* accel;          // [n_part][3]
    double* pot;            // [n_part]
};

// Stages cnt entries buf[0..cnt) (cells: source n_part + k, else particles)
// as pair records relative to the group centre c and evaluates them for the
// lane's IB targets; the tile sums go into the Kahan sums acc.
template <int IB>
__device__ __forceinline__ void fuse_tile(const WalkArgs& a, const FuseArgs& f, const int32_t* buf, int cnt, bool cell,
                                          float4* rec, int lane, int nsub, int js, bool active, float cx, float cy,
                                          float cz, const f2 nx[IB], const f2 ny[IB], const f2 nz[IB], f2 e2,
                                          float eps2, Acc<float> acc[IB], uint32_t* status)
{
    const bool cq = cell && f.quad != nullptr;
    const int npair = (cnt + 1) / 2;
    const int npair_pad = (npair + nsub - 1) / nsub * nsub;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t n_src = a.n_part + a.n_cell;
#pragma unroll
    for (int pp = 0; pp < kFusePPL; ++pp) {
        const int m = lane + 32 * pp;
        if (m >= npair_pad) continue;
        float4 hh[2], ll[2], qa[2], qb[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * m + h;
            hh[h] = ll[h] = qa[h] = qb[h] = zero4;
            if (k < cnt) {
                const int idx = buf[k];
                const bool good = cell ? (idx >= a.n_part && idx < n_src) : (idx >= 0 && idx < a.n_part);
                if (good) {
                    hh[h] = __ldg(f.split + 2 * (int64_t)idx);
                    ll[h] = __ldg(f.split + 2 * (int64_t)idx + 1);
                    if (cq) {
                        const float4* qp = reinterpret_cast<const float4*>(f.quad + (idx - a.n_part));
                        qa[h] = __ldg(qp);
                        qb[h] = __ldg(qp + 1);
                    }
                } else {
                    atomicOr(status, kWalkBadRecord);
                }
            }
        }
        // padding and rejected entries were loaded as zeros: mass (and
        // quadrupole) 0, so they add exactly nothing
        float x[2], y[2], z[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            x[h] = rel32(hh[h].x, ll[h].x, cx);
            y[h] = rel32(hh[h].y, ll[h].y, cy);
            z[h] = rel32(hh[h].z, ll[h].z, cz);
        }
        const float w[2] = {hh[0].w, hh[1].w};
        put_rec2(rec, m, cq, x, y, z, w, qa, qb, eps2);
    }
    __syncwarp();
    if (active) {
        const f2 zero2 = f2pack(0.f, 0.f);
        Acc2 P2[IB];
#pragma unroll
        for (int k = 0; k < IB; ++k) P2[k].v[0] = P2[k].v[1] = P2[k].v[2] = P2[k].v[3] = zero2;
        const int niter = npair_pad / nsub;
        // loops not unrolled: the walk and the evaluation alternate in one
        // warp and must fit the instruction cache together
        if (cq)
            eval_cells2<IB, 1>(rec, js, nsub, niter, nx, ny, nz, e2, P2);
        else
            eval_parts2<IB, 1>(rec, js, nsub, niter, nx, ny, nz, e2, P2);
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            float t4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float lo, hi;
                f2unpack(P2[k].v[c], lo, hi);
                t4[c] = lo + hi;
            }
            acc[k].add(t4);
        }
    }
    __syncwarp();
}

// Drops the first `used` entries of buf (n in total; n - used < used).
__device__ __forceinline__ void fuse_shift(int32_t* buf, int n, int used, int lane)
{
    for (int k = lane; k < n - used; k += 32) buf[k] = buf[used + k];
    __syncwarp();
}

template <int IB>
#ifndef OTOO_FUSE_MIN_BLOCKS
#define OTOO_FUSE_MIN_BLOCKS 3  // resident CTAs per SM asked of the register allocator (168 registers)
#endif
__global__ void __launch_bounds__(kFuseWarps * 32, OTOO_FUSE_MIN_BLOCKS) k_walk_force(WalkArgs a, FuseArgs f)
{
    __shared__ uint32_t stack_s[kFuseWarps][kStack];
    __shared__ int32_t cbuf_s[kFuseWarps][kFuseBuf];
    __shared__ int32_t pbuf_s[kFuseWarps][kFuseBuf];
    __shared__ float4 rec_s[kFuseWarps][kCellRecF4 * kFuseTP];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint32_t* stk = stack_s[wid];
    int32_t* cbuf = cbuf_s[wid];
    int32_t* pbuf = pbuf_s[wid];
    float4* rec = rec_s[wid];
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* status = a.counter + 1;
    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(a.counter, 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= a.n_groups) break;
        const int32_t first = a.gfirst[g], count = a.gcount[g];
        if (first < 0 || count < 1 || count > 32 * IB || (int64_t)first + count > a.n_part) {
            if (lane == 0) atomicOr(status, kWalkBadGroup);
            continue;
        }
        GroupWalk w;
        group_walk_setup(a, g, first, count, lane, w);
        if (!(w.theta >= 0.0)) continue;  // a negative per-group angle skips the group

        // the group's particles, IB per lane in nsub lane subsets
        const int P = (count + IB - 1) / IB;
        const int nsub = 32 / P;
        const int islot = lane % P, js = lane / P;
        const bool active = js < nsub;
        // entries per evaluated tile: a multiple of 2 nsub
        const int TE = 2 * ((kFuseTP / nsub) * nsub);
        const float eps2 = (float)a.eps2;
        const f2 e2 = f2pack(eps2, eps2);
        const float cx = __double2float_rn(w.c[0]), cy = __double2float_rn(w.c[1]), cz = __double2float_rn(w.c[2]);
        f2 nx[IB], ny[IB], nz[IB];
        Acc<float> acc[IB];
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            const int i = islot + k * P;
            float x = 0.f, y = 0.f, z = 0.f;
            if (active && i < count) {
                const int64_t t = (int64_t)first + i;
                const float4 h = __ldg(f.split + 2 * t);
                const float4 l = __ldg(f.split + 2 * t + 1);
                x = rel32(h.x, l.x, cx);
                y = rel32(h.y, l.y, cy);
                z = rel32(h.z, l.z, cz);
            }
            nx[k] = f2pack(-x, -x);
            ny[k] = f2pack(-y, -y);
            nz[k] = f2pack(-z, -z);
            acc[k].zero();
        }

        int32_t ncell = 0, npart = 0;  // entries of the group's (virtual) list
        int nc = 0, npb = 0;           // entries waiting in the two buffers
        int sp = 1;
        if (lane == 0) stk[0] = run(0, 1);
        __syncwarp();
        int64_t budget = a.n_cell;
        bool failed = false;
        while (sp > 0) {
            StepCells sc;
            if (!walk_take(a, w, stk, sp, budget, lane, sc, status)) {
                failed = true;
                break;
            }
            // accepted cells into the cell buffer, in position order
#pragma unroll
            for (int h = 0; h < kWalkHalves; ++h) {
                const unsigned am = __ballot_sync(kFull, sc.kind[h] == 1);
                if (sc.kind[h] == 1) cbuf[nc + __popc(am & lt)] = (int32_t)(a.n_part + sc.node[h]);
                nc += __popc(am);
                ncell += __popc(am);
            }
            __syncwarp();
            // particles of rejected leaves into the particle buffer, in
            // position order, a buffer's worth at a time
#pragma unroll
            for (int h = 0; h < kWalkHalves; ++h) {
                if (!__any_sync(kFull, sc.kind[h] == 2)) continue;
                const int np = sc.kind[h] == 2 ? sc.pe[h] - sc.pb[h] : 0;
                const int pin = warp_incl_scan(np, lane);
                const int total = __shfl_sync(kFull, pin, 31);
                npart += total;
                for (int done = 0; done < total;) {
                    const int take = min(kFuseBuf - npb, total - done);
                    const int lo = max(pin - np, done), hi = min(pin, done + take);
                    for (int o = lo; o < hi; ++o) pbuf[npb + o - done] = sc.pb[h] + (o - (pin - np));
                    __syncwarp();
                    npb += take;
                    done += take;
                    while (npb >= TE) {
                        fuse_tile<IB>(a, f, pbuf, TE, false, rec, lane, nsub, js, active, cx, cy, cz, nx, ny, nz, e2,
                                      eps2, acc, status);
                        fuse_shift(pbuf, npb, TE, lane);
                        npb -= TE;
                    }
                }
            }
            walk_push(stk, sp, sc, lt);
            while (nc >= TE) {
                fuse_tile<IB>(a, f, cbuf, TE, true, rec, lane, nsub, js, active, cx, cy, cz, nx, ny, nz, e2, eps2, acc,
                              status);
                fuse_shift(cbuf, nc, TE, lane);
                nc -= TE;
            }
        }
        if (failed) {
            if (lane == 0) atomicOr(status, kWalkOverflow);
            continue;
        }
        if (nc > 0)
            fuse_tile<IB>(a, f, cbuf, nc, true, rec, lane, nsub, js, active, cx, cy, cz, nx, ny, nz, e2, eps2, acc, status);
        if (npb > 0)
            fuse_tile<IB>(a, f, pbuf, npb, false, rec, lane, nsub, js, active, cx, cy, cz, nx, ny, nz, e2, eps2, acc,
                          status);

        // merge the lane subsets, FP64 outputs in caller order; the self pair
        // (always in the list: a group never accepts a cell overlapping its
        // box) added exactly -m_i rsqrt(eps^2) in FP32
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            double r[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float S = acc[k].s[c], C = acc[k].c[c];
                merge_subsets(S, C, js, nsub, P);
                r[c] = (double)S - (double)C;
            }
            r[3] = -r[3];
            const int i = islot + k * P;
            if (js == 0 && i < count) {
                const int64_t t = (int64_t)first + i;
                const float4 h = __ldg(f.split + 2 * t);
                r[3] += (double)(h.w * rsqrt_r(eps2));
                const int64_t o = f.perm ? f.perm[t] : t;
                f.accel[3 * o] = r[0];
                f.accel[3 * o + 1] = r[1];
                f.accel[3 * o + 2] = r[2];
                f.pot[o] = r[3];
            }
        }
        if (lane == 0) {
            const int64_t len = (int64_t)ncell + npart;
            atomicAdd(reinterpret_cast<unsigned long long*>(a.totals), (unsigned long long)len);
            atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 1), (unsigned long long)(len * count));
            atomicAdd(reinterpret_cast<unsigned long long*>(a.totals + 2), (unsigned long long)((int64_t)ncell * count));
            atomicMax(reinterpret_cast<unsigned long long*>(a.totals + 3), (unsigned long long)ncell);
            atomicMax(reinterpret_cast<unsigned long long*>(a.totals + 4), (unsigned long long)npart);
        }
    }
}

// One warp per group: the group's slot (filled by the single pass) copied to
// its place in the dense list (list_off, already rewritten by the scan),
// cells back in walk order, then particles.  Nothing is copied when a group
// did not fit its slot (totals[5] > 0: the caller walks again in two passes)
// or when the list is too small.
__global__ void k_compact(const otoo_group* __restrict__ groups, int32_t G, const int32_t* __restrict__ slots,
                          int64_t ccap, int64_t pcap, int32_t* __restrict__ list, int64_t capacity,
                          const int64_t* __restrict__ totals, uint32_t* __restrict__ status)
{
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= G) return;
    if (totals[5] > 0 || totals[0] > capacity) {
        if (g == 0 && lane == 0) atomicOr(status, kWalkNoRoom);
        return;
    }
    const otoo_group gr = groups[g];
    if (gr.n_cell < 0 || gr.n_part < 0 || gr.n_cell > ccap || gr.n_part > pcap || gr.list_off < 0 ||
        gr.list_off + gr.n_cell + gr.n_part > capacity) {
        if (lane == 0) atomicOr(status, kWalkNoRoom);
        return;
    }
    const int32_t* ps = slots + g * (ccap + pcap) + ccap;  // particle 0; cell k at ps[-1 - k]
    int32_t* d = list + gr.list_off;
    for (int k = lane; k < gr.n_cell; k += 32) d[k] = ps[-1 - k];
    d += gr.n_cell;
    for (int k = lane; k < gr.n_part; k += 32) d[k] = ps[k];
}

// ---- exclusive prefix sums in index order ---------------------------------
// In: functor int64 operator()(int64 i); Out: functor void operator()(int64 i,
// int64 prefix).  Three launches: sums of blocks of kScanBlock elements, a
// one-CTA exclusive scan of those sums (total to *total), block-level scans.

struct GroupLen {
    const otoo_group* g;
    __device__ int64_t operator()(int64_t i) const { return (int64_t)g[i].n_cell + g[i].n_part; }
};
struct GroupOff {
    otoo_group* g;
    __device__ void operator()(int64_t i, int64_t v) const { g[i].list_off = v; }
};
struct I32In {
    const int32_t* p;
    __device__ int64_t operator()(int64_t i) const { return p[i]; }
};
struct I32Out {
    int32_t* p;
    __device__ void operator()(int64_t i, int64_t v) const { p[i] = (int32_t)v; }
};

__device__ int64_t block_excl_scan(int64_t v, int64_t* warp_s, int64_t* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_s[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? warp_s[lane] : 0;
        int64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        warp_s[lane] = wi - w;
        if (lane == 31) warp_s[32] = wi;
    }
    __syncthreads();
    const int64_t r = warp_s[wid] + inc - v;
    *total = warp_s[32];
    __syncthreads();
    return r;
}

template <class In>
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(In in, int64_t n, int64_t* __restrict__ bsum)
{
    __shared__ int64_t ws[33];
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
    int64_t v = 0;
    for (int k = 0; k < kScanBlock / kScanThreads; ++k) {
        const int64_t i = b0 + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < n) v += in(i);
    }
    int64_t tot;
    block_excl_scan(v, ws, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int64_t* __restrict__ bsum, int64_t nblk,
                                                            int64_t* __restrict__ total)
{
    __shared__ int64_t ws[33];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nblk; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        const int64_t v = i < nblk ? bsum[i] : 0;
        int64_t tot;
        const int64_t e = block_excl_scan(v, ws, &tot);
        if (i < nblk) bsum[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <class In, class Out>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(In in, Out out, int64_t n,
                                                              const int64_t* __restrict__ bsum)
{
    __shared__ int64_t ws[33];
    constexpr int kPer = kScanBlock / kScanThreads;
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kPer;
    int64_t v[kPer], s = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = b0 + k < n ? in(b0 + k) : 0;
        s += v[k];
    }
    int64_t tot;
    int64_t e = block_excl_scan(s, ws, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (b0 + k < n) out(b0 + k, e);
        e += v[k];
    }
}

template <class In, class Out>
cudaError_t excl_scan(In in, Out out, int64_t n, int64_t* bsum, int64_t* total, cudaStream_t s)
{
    const int64_t nblk = (n + kScanBlock - 1) / kScanBlock;
    if (nblk == 0) return cudaSuccess;
    k_scan_sums<In><<<(unsigned)nblk, kScanThreads, 0, s>>>(in, n, bsum);
    k_scan_top<<<1, kScanThreads, 0, s>>>(bsum, nblk, total);
    k_scan_apply<In, Out><<<(unsigned)nblk, kScanThreads, 0, s>>>(in, out, n, bsum);
    return cudaGetLastError();
}

int64_t scan_blocks(int64_t n) { return (n + kScanBlock - 1) / kScanBlock; }

// ---- device plan ------------------------------------------------------------

struct PlanScratch {
    int64_t* bsum;    // scan block sums (2 scans, one after the other)
    int32_t* hist;    // [kClasses] items per cost class
    int32_t* cursor;  // [kClasses] next free item position of each class
    int32_t* nic;     // [G] particle chunks
    int32_t* nch;     // [G] list chunks
    int32_t* slot0;   // [G] slots (n_chunks when > 1), then their exclusive prefix
    int32_t* sidx;    // [G] 1 when the list is split, then the split record index
    int32_t* cls;     // [G] cost class
};

PlanScratch plan_layout(int32_t* base, int64_t G)
{
    PlanScratch p;
    const int64_t nb = scan_blocks(G) + 1;
    p.bsum = reinterpret_cast<int64_t*>(base);
    int32_t* q = base + 2 * nb;
    p.hist = q;
    p.cursor = q + kClasses;
    q += 2 * kClasses;
    p.nic = q;
    p.nch = q + G;
    p.slot0 = q + 2 * G;
    p.sidx = q + 3 * G;
    p.cls = q + 4 * G;
    return p;
}

// The plan kernels run 256 threads per block, one group each.  The chunk
// table (a kernel parameter) is copied to shared memory first: threads index
// it by their own group sizes, which the parameter bank would serialise.
// Counts and totals are summed per block in shared memory, so each block
// makes one global atomic per class and per total instead of one per group.
constexpr int kPlanThreads = 256;

__device__ void plan_table_to_shared(const ChunkTable& tab, ChunkTable& st)
{
    for (int k = threadIdx.x; k <= kMaxGroup; k += blockDim.x) st.last[k] = tab.last[k];
    if (threadIdx.x == 0) st.ib = tab.ib;
}

__global__ void __launch_bounds__(kPlanThreads) k_plan_count(const otoo_group* __restrict__ groups, int32_t G,
                                                             const ChunkTable tab, int32_t split, PlanScratch p,
                                                             int64_t* __restrict__ totals)
{
    __shared__ ChunkTable st;
    __shared__ int32_t shist[kClasses];
    __shared__ unsigned long long s_items, s_split_groups, s_split_chunks, s_max;
    plan_table_to_shared(tab, st);
    for (int c = threadIdx.x; c < kClasses; c += blockDim.x) shist[c] = 0;
    if (threadIdx.x == 0) s_items = s_split_groups = s_split_chunks = s_max = 0;
    __syncthreads();
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < G) {
        const otoo_group gr = groups[g];
        atomicMax(&s_max, (unsigned long long)(gr.count > 1 ? gr.count : 1));
        const int64_t len = (int64_t)gr.n_cell + gr.n_part;
        int32_t nic = 0, nch = 0, cls = 0;
        if (len > 0 && gr.count > 0 && gr.count <= kMaxGroup) {
            // the host plan's particle chunks (plan_chunks.h)
            int32_t big = 0;
            nic = chunk_count(st, gr.count, &big);
            nch = (int32_t)((len + split - 1) / split);
            // cost class: 4 * log2 of the largest item's ni * (j1 - j0), in quarter octaves
            const int64_t c0 = (int64_t)big * ((len + nch - 1) / nch);
            const int msb = 63 - __clzll((long long)c0);
            const int frac = msb >= 2 ? (int)((c0 >> (msb - 2)) & 3) : (int)((c0 << (2 - msb)) & 3);
            cls = 4 * msb + frac;
            if (cls >= kClasses) cls = kClasses - 1;
            atomicAdd(shist + cls, nic * nch);
            atomicAdd(&s_items, (unsigned long long)(nic * nch));
            if (nch > 1) {
                atomicAdd(&s_split_groups, 1ull);
                atomicAdd(&s_split_chunks, (unsigned long long)nch);
            }
        }
        p.nic[g] = nic;
        p.nch[g] = nch;
        p.slot0[g] = nch > 1 ? nch : 0;
        p.sidx[g] = nch > 1 ? 1 : 0;
        p.cls[g] = cls;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < kClasses; c += blockDim.x)
        if (shist[c]) atomicAdd(p.hist + c, shist[c]);
    if (threadIdx.x == 0) {
        unsigned long long* t = reinterpret_cast<unsigned long long*>(totals);
        if (s_items) atomicAdd(t, s_items);
        if (s_split_groups) {
            atomicAdd(t + 1, s_split_groups);
            atomicAdd(t + 2, s_split_chunks);
        }
        atomicMax(t + 3, s_max);
    }
}

__global__ void k_plan_cursor(PlanScratch p)
{
    if (threadIdx.x != 0) return;
    int32_t pos = 0;
    for (int c = kClasses - 1; c >= 0; --c) {
        p.cursor[c] = pos;
        pos += p.hist[c];
    }
}

__global__ void __launch_bounds__(kPlanThreads) k_plan_fill(const otoo_group* __restrict__ groups, int32_t G,
                                                            const ChunkTable tab, PlanScratch p,
                                                            otoo_item* __restrict__ items, int64_t items_cap,
                                                            otoo_split* __restrict__ splits, int64_t splits_cap,
                                                            uint32_t* __restrict__ status)
{
    __shared__ ChunkTable st;
    __shared__ int32_t scount[kClasses], sbase[kClasses];
    plan_table_to_shared(tab, st);
    for (int c = threadIdx.x; c < kClasses; c += blockDim.x) scount[c] = 0;
    __syncthreads();
    // the block's items of each class take one run of that class's items
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t nic = g < G ? p.nic[g] : 0, nch = g < G ? p.nch[g] : 0;
    const bool on = nic > 0 && nch > 0;
    const int32_t cls = on ? p.cls[g] : 0;
    const int32_t local = on ? atomicAdd(scount + cls, nic * nch) : 0;
    __syncthreads();
    for (int c = threadIdx.x; c < kClasses; c += blockDim.x)
        if (scount[c]) sbase[c] = atomicAdd(p.cursor + c, scount[c]);
    __syncthreads();
    if (!on) return;
    const otoo_group gr = groups[g];
    const int64_t len = (int64_t)gr.n_cell + gr.n_part;
    const int32_t slot0 = p.slot0[g];
    const int32_t pos = sbase[cls] + local;
    if ((int64_t)pos + nic * nch > items_cap) {
        atomicOr(status, kWalkNoRoom);
        return;
    }
    if (nch > 1) {
        const int32_t si = p.sidx[g];
        if (si >= splits_cap) {
            atomicOr(status, kWalkNoRoom);
            return;
        }
        otoo_split s;
        s.g = g;
        s.slot0 = slot0;
        s.n_chunks = nch;
        s.pad = 0;
        splits[si] = s;
    }
    int32_t k = pos, i0 = 0;
    for (int32_t rest = gr.count; rest > 0;) {
        const int32_t ni = st.last[rest];
        for (int32_t q = 0; q < nch; ++q) {
            otoo_item it;
            it.g = g;
            it.i0 = i0;
            it.ni = ni;
            it.j0 = (int32_t)(len * q / nch);
            it.j1 = (int32_t)(len * (q + 1) / nch);
            it.slot = nch > 1 ? slot0 + q : -1;
            it.pad0 = it.pad1 = 0;
            items[k++] = it;
        }
        i0 += ni;
        rest -= ni;
    }
}

#define CUDA_TRY(expr)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return set_error(OTOO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

// The particle-chunk table of the plan for ib targets per lane, built once
// per process for each ib in {1, 2, 4} (others each call).
const ChunkTable& chunk_table(int32_t ib)
{
    static ChunkTable tabs[3];
    static std::once_flag once[3];
    const int k = ib == 1 ? 0 : ib == 2 ? 1 : ib == 4 ? 2 : -1;
    if (k < 0) {
        thread_local ChunkTable t;
        chunk_table_build(ib, t);
        return t;
    }
    std::call_once(once[k], [&] { chunk_table_build(ib, tabs[k]); });
    return tabs[k];
}

int check_walk(const otoo_dev_walk* w)
{
    OTOO_REQUIRE(w, OTOO_EINVAL, "walk is NULL");
    OTOO_REQUIRE(w->src && w->cell && w->cell64 && w->group_first && w->group_count && w->counter && w->totals,
                 OTOO_EINVAL, "walk: NULL device pointer");
    OTOO_REQUIRE(w->n_part >= 1 && w->n_cell >= 1 && w->n_part + w->n_cell <= INT32_MAX, OTOO_EINVAL,
                 "walk: n_part/n_cell out of range");
    OTOO_REQUIRE(w->n_cell <= (int64_t)kRunMask + 1, OTOO_EINVAL, "walk: more than 2^28 cells");
    OTOO_REQUIRE(w->n_groups >= 1, OTOO_EINVAL, "walk: n_groups < 1");
    OTOO_REQUIRE(w->eps2 > 0.0, OTOO_EINVAL, "walk: eps2 must be > 0");
    OTOO_REQUIRE(w->theta >= 0.0 && w->theta < 1e300, OTOO_EINVAL, "walk: theta must be finite and >= 0");
    OTOO_REQUIRE(w->set >= 0 && w->set <= kSet, OTOO_EINVAL, "walk: set must be in [0, %d]", kSet);
    OTOO_REQUIRE(w->mac == OTOO_MAC_THETA || w->mac == OTOO_MAC_SW || w->mac == OTOO_MAC_SPH, OTOO_EINVAL,
                 "walk: unknown mac %d", w->mac);
    return OTOO_OK;
}

WalkArgs walk_args(const otoo_dev_walk* w)
{
    WalkArgs a;
    a.n_part = w->n_part;
    a.n_cell = w->n_cell;
    a.n_groups = w->n_groups;
    a.exact = w->exact ? 1 : 0;
    a.mac = w->mac;
    a.pad = 0;
    a.theta = w->theta;
    a.eps2 = w->eps2;
    a.src = w->src;
    a.cell = w->cell;
    a.cell64 = w->cell64;
    a.gfirst = w->group_first;
    a.gcount = w->group_count;
    a.tpg = w->theta_per_group;
    a.counter = w->counter;
    a.totals = w->totals;
    return a;
}

template <int kMode>
int launch_walk(const otoo_dev_walk* w, otoo_group* groups, int32_t* list, int64_t capacity, cudaStream_t s,
                int64_t pcap = 0)
{
    int dev = 0, sms = 0, occ = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // groups per warp: as asked, or (0) up to kSet while every resident warp
    // still gets about three sets to balance the load
    int gs = w->set;
    if (gs == 0) {
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_walk_set<kMode>, kWalkWarps * 32, 0));
        const int64_t warps = (int64_t)sms * (occ < 1 ? 1 : occ) * kWalkWarps;
        const int64_t fit = (int64_t)w->n_groups / (3 * warps);
        gs = fit < 1 ? 1 : fit > kSet ? kSet : (int)fit;
    }
    const bool sets = gs > 1;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, sets ? (const void*)k_walk_set<kMode> : (const void*)k_walk<kMode>, kWalkWarps * 32, 0));
    if (occ < 1) occ = 1;
    int64_t blocks = (int64_t)sms * occ;
    const int64_t units = ((int64_t)w->n_groups + gs - 1) / gs;
    const int64_t need = (units + kWalkWarps - 1) / kWalkWarps;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    CUDA_TRY(cudaMemsetAsync(w->counter, 0, sizeof(uint32_t), s));
    if (sets)
        k_walk_set<kMode><<<(unsigned)blocks, kWalkWarps * 32, 0, s>>>(walk_args(w), (int32_t)units, gs, groups,
                                                                      list, capacity, pcap);
    else
        k_walk<kMode><<<(unsigned)blocks, kWalkWarps * 32, 0, s>>>(walk_args(w), groups, list, capacity, pcap);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

}  // namespace

extern "C" {

int64_t otoo_walk_totals_len(int64_t n_groups) { return kTotals + scan_blocks(n_groups < 0 ? 0 : n_groups) + 1; }

int otoo_walk_count(const otoo_dev_walk* w, otoo_group* groups, void* stream)
{
    otoo::Range range_("otoo_walk_count");
    const int rc = check_walk(w);
    if (rc) return rc;
    OTOO_REQUIRE(groups, OTOO_EINVAL, "otoo_walk_count: groups is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(w->counter, 0, 4 * sizeof(uint32_t), s));
    CUDA_TRY(cudaMemsetAsync(w->totals, 0, kTotals * sizeof(int64_t), s));
    const int r2 = launch_walk<0>(w, groups, nullptr, 0, s);
    if (r2) return r2;
    CUDA_TRY(excl_scan(GroupLen{groups}, GroupOff{groups}, w->n_groups, w->totals + kTotals, nullptr, s));
    return OTOO_OK;
}

int otoo_walk_single(const otoo_dev_walk* w, otoo_group* groups, int32_t* slots, int64_t cell_cap, int64_t part_cap,
                     void* stream)
{
    otoo::Range range_("otoo_walk_single");
    const int rc = check_walk(w);
    if (rc) return rc;
    OTOO_REQUIRE(groups && slots, OTOO_EINVAL, "otoo_walk_single: NULL pointer");
    OTOO_REQUIRE(cell_cap >= 1 && part_cap >= 1 && cell_cap + part_cap <= INT32_MAX, OTOO_EINVAL,
                 "otoo_walk_single: slot sizes out of range");
    OTOO_REQUIRE(w->n_groups <= INT64_MAX / (cell_cap + part_cap), OTOO_EINVAL, "otoo_walk_single: slots too large");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(w->counter, 0, 4 * sizeof(uint32_t), s));
    CUDA_TRY(cudaMemsetAsync(w->totals, 0, kTotals * sizeof(int64_t), s));
    return launch_walk<2>(w, groups, slots, cell_cap, s, part_cap);
}

int otoo_walk_compact(const otoo_dev_walk* w, otoo_group* groups, const int32_t* slots, int64_t cell_cap,
                      int64_t part_cap, int32_t* list, int64_t capacity, void* stream)
{
    otoo::Range range_("otoo_walk_compact");
    const int rc = check_walk(w);
    if (rc) return rc;
    OTOO_REQUIRE(groups && slots && list, OTOO_EINVAL, "otoo_walk_compact: NULL pointer");
    OTOO_REQUIRE(cell_cap >= 1 && part_cap >= 1 && cell_cap + part_cap <= INT32_MAX, OTOO_EINVAL,
                 "otoo_walk_compact: slot sizes out of range");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(excl_scan(GroupLen{groups}, GroupOff{groups}, w->n_groups, w->totals + kTotals, nullptr, s));
    const int64_t warps = w->n_groups;
    k_compact<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(groups, w->n_groups, slots, cell_cap, part_cap,
                                                                   list, capacity, w->totals, w->counter + 1);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int otoo_walk_fill(const otoo_dev_walk* w, const otoo_group* groups, int32_t* list, int64_t capacity, void* stream)
{
    otoo::Range range_("otoo_walk_fill");
    const int rc = check_walk(w);
    if (rc) return rc;
    OTOO_REQUIRE(groups && list, OTOO_EINVAL, "otoo_walk_fill: NULL pointer");
    OTOO_REQUIRE(capacity >= 0, OTOO_EINVAL, "otoo_walk_fill: negative capacity");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return launch_walk<1>(w, const_cast<otoo_group*>(groups), list, capacity, s);
}

int otoo_walk_force(const otoo_dev_walk* w, const otoo_quad* quad, const int64_t* perm, float* split, int32_t iblock,
                    double* accel, double* pot, void* stream)
{
    otoo::Range range_("otoo_walk_force");
    const int rc = check_walk(w);
    if (rc) return rc;
    OTOO_REQUIRE(split && accel && pot, OTOO_EINVAL, "otoo_walk_force: NULL pointer");
    OTOO_REQUIRE(w->mac != OTOO_MAC_SPH, OTOO_EINVAL, "otoo_walk_force: the SPH walk has no force");
    OTOO_REQUIRE(iblock == 1 || iblock == 2 || iblock == 4, OTOO_EINVAL, "otoo_walk_force: iblock must be 1, 2 or 4");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(w->counter, 0, 4 * sizeof(uint32_t), s));
    CUDA_TRY(cudaMemsetAsync(w->totals, 0, kTotals * sizeof(int64_t), s));
    const int r1 = enqueue_split(w->src, split, w->n_part + w->n_cell, stream);
    if (r1) return r1;
    FuseArgs f;
    f.split = reinterpret_cast<const float4*>(split);
    f.quad = quad;
    f.perm = perm;
    f.accel = accel;
    f.pot = pot;
    void (*fn)(WalkArgs, FuseArgs) = iblock == 1 ? k_walk_force<1> : iblock == 2 ? k_walk_force<2> : k_walk_force<4>;
    int dev = 0, sms = 0, occ = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kFuseWarps * 32, 0));
    if (occ < 1) return set_error(OTOO_EINVAL, "otoo_walk_force: kernel does not fit on an SM");
    int64_t blocks = (int64_t)sms * occ;
    const int64_t need = ((int64_t)w->n_groups + kFuseWarps - 1) / kFuseWarps;
    if (blocks > need) blocks = need;
    fn<<<(unsigned)blocks, kFuseWarps * 32, 0, s>>>(walk_args(w), f);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int otoo_walk_check_status(const otoo_dev_walk* w, void* stream)
{
    OTOO_REQUIRE(w && w->counter, OTOO_EINVAL, "walk/counter is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t h[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(h, w->counter, sizeof(h), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (h[1] & kWalkBadGroup) return set_error(OTOO_EDEVICE, "walk: a group range failed its bounds check");
    if (h[1] & kWalkBadRecord) return set_error(OTOO_EDEVICE, "walk: a cell record failed its bounds check");
    if (h[1] & kWalkOverflow) return set_error(OTOO_EDEVICE, "walk: a group's stack or node budget ran out");
    if (h[1] & kWalkMismatch) return set_error(OTOO_EDEVICE, "walk: the two passes counted different entries");
    if (h[1] & kWalkNoRoom) return set_error(OTOO_EDEVICE, "walk/plan: output array too small");
    return OTOO_OK;
}

int64_t otoo_plan_scratch_ints(int64_t n_groups)
{
    if (n_groups < 0) n_groups = 0;
    return 2 * (scan_blocks(n_groups) + 1) + 2 * kClasses + 5 * n_groups;
}

int otoo_plan_count(const otoo_group* groups, int32_t n_groups, const otoo_tune* tune, int32_t* plan_scratch,
                    int64_t* plan_totals, void* stream)
{
    otoo::Range range_("otoo_plan_count");
    OTOO_REQUIRE(groups && tune && plan_scratch && plan_totals, OTOO_EINVAL, "otoo_plan_count: NULL pointer");
    OTOO_REQUIRE(n_groups >= 1, OTOO_EINVAL, "otoo_plan_count: n_groups < 1");
    OTOO_REQUIRE(tune->split >= 1, OTOO_EINVAL, "split must be >= 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int32_t ib = tune->iblock > 1 ? tune->iblock : 1;
    PlanScratch p = plan_layout(plan_scratch, n_groups);
    CUDA_TRY(cudaMemsetAsync(plan_totals, 0, 4 * sizeof(int64_t), s));
    CUDA_TRY(cudaMemsetAsync(p.hist, 0, kClasses * sizeof(int32_t), s));
    k_plan_count<<<(n_groups + kPlanThreads - 1) / kPlanThreads, kPlanThreads, 0, s>>>(
        groups, n_groups, chunk_table(ib), tune->split, p, plan_totals);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(excl_scan(I32In{p.slot0}, I32Out{p.slot0}, n_groups, p.bsum, nullptr, s));
    CUDA_TRY(excl_scan(I32In{p.sidx}, I32Out{p.sidx}, n_groups, p.bsum, nullptr, s));
    k_plan_cursor<<<1, 32, 0, s>>>(p);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

int otoo_plan_fill(const otoo_group* groups, int32_t n_groups, const otoo_tune* tune, int32_t* plan_scratch,
                   const int64_t* plan_totals, otoo_item* items, int64_t items_capacity, otoo_split* splits,
                   int64_t splits_capacity, uint32_t* counter, void* stream)
{
    otoo::Range range_("otoo_plan_fill");
    OTOO_REQUIRE(groups && tune && plan_scratch && plan_totals && counter, OTOO_EINVAL,
                 "otoo_plan_fill: NULL pointer");
    OTOO_REQUIRE(items || items_capacity == 0, OTOO_EINVAL, "otoo_plan_fill: items is NULL");
    OTOO_REQUIRE(splits || splits_capacity == 0, OTOO_EINVAL, "otoo_plan_fill: splits is NULL");
    OTOO_REQUIRE(n_groups >= 1, OTOO_EINVAL, "otoo_plan_fill: n_groups < 1");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int32_t ib = tune->iblock > 1 ? tune->iblock : 1;
    PlanScratch p = plan_layout(plan_scratch, n_groups);
    k_plan_fill<<<(n_groups + kPlanThreads - 1) / kPlanThreads, kPlanThreads, 0, s>>>(
        groups, n_groups, chunk_table(ib), p, items, items_capacity, splits, splits_capacity, counter + 1);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

}  // extern "C"
