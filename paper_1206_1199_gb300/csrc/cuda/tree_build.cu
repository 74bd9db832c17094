// The octree built on the device (Section III-B: root cube, keys, sort,
// cells; Section III-C: cell properties), producing the inputs of the device
// walk and the force step directly in device memory.
//
// The root cube, the grid coordinates, the Hilbert keys and the cube of every
// cell are computed with the host build's operations (treegeom.h), and the
// sort is stable on (key, caller index), so the particle order, the cells (as
// (level, first particle, last particle) ranges), their cubes and the groups
// are the host build's.  Cells are numbered level by level (the host numbers
// them in expansion order); children stay consecutive.  Moments are summed
// bottom-up (children combined by the parallel-axis rule), so they equal the
// host's direct sums to rounding.
//
// Kernels
//   k_bbox / k_bbox_final   min/max of the positions (order-preserving integer
//                           keys: exact), then the root cube.
//   k_keys                  grid coordinates and Hilbert key per particle.
//   k_rs_hist / k_rs_scatter  stable LSD radix sort of (key, index), 8 bits
//                           per pass: per-block digit counts, a scan of the
//                           counts (digit-major), a scatter that ranks equal
//                           digits in input order (warp match + per-warp
//                           running counts).
//   k_permute               particles in tree order (sources, permutation,
//                           grid coordinates).
//   k_expand_count / k_expand_write  one level of cells from the previous one:
//                           a cell with more than leaf_size particles (above
//                           the last grid level) splits into the runs of its
//                           particles' next key digit, found by binary search.
//   k_moments               leaves sum their particles (all leaves in one
//                           launch), then parents combine their children, one
//                           level per launch, deepest first.
//   k_bmax                  largest distance of a cell's particles from its
//                           centre of mass (FP64, on the particles an FP32
//                           bound leaves), or the SPH radius bound (FP32);
//                           chunks of particles, atomic max.
//   k_records               sources, quadrupoles and walk records of the cells.
//   k_group_flags           first particle of every group (maximal cells with
//                           at most n_crit particles; larger leaves in chunks).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "../common.h"
#include "../treegeom.h"

using namespace otoo;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRsThreads = 256;                 // radix sort: threads per block
constexpr int kRsItems = 8;                     // keys per thread
constexpr int kRsTile = kRsThreads * kRsItems;  // keys per block
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kBmaxChunk = 2048;                // particles per b_max work item

// status bits
constexpr uint32_t kTreeBadInput = 1u;   // a non-finite position or a mass <= 0
constexpr uint32_t kTreeBadSort = 2u;    // the sorted order indexed outside the particles

struct Geom {
    double lo[3], S, h, scale;
};

__device__ __forceinline__ long long dkey(double x)
{
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dval(long long k) { return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL)); }

// ---- bounding box ------------------------------------------------------------

__global__ void __launch_bounds__(256) k_bbox(const double* __restrict__ pos, const float* __restrict__ mass, int64_t n,
                                              long long* __restrict__ part, uint32_t* __restrict__ status)
{
    long long lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = 0x7fffffffffffffffLL, hi[a] = -lo[a] - 1;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            const double x = pos[3 * i + a];
            bad |= !isfinite(x);
            const long long k = dkey(x);
            lo[a] = k < lo[a] ? k : lo[a];
            hi[a] = k > hi[a] ? k : hi[a];
        }
        const float m = mass[i];
        bad |= !(m > 0.0f) || !isfinite(m);
    }
    if (bad) atomicOr(status, kTreeBadInput);
    __shared__ long long s[6][8];
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            const long long t0 = __shfl_xor_sync(kFull, lo[a], o), t1 = __shfl_xor_sync(kFull, hi[a], o);
            lo[a] = t0 < lo[a] ? t0 : lo[a];
            hi[a] = t1 > hi[a] ? t1 : hi[a];
        }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) s[a][w] = lo[a], s[3 + a][w] = hi[a];
    __syncthreads();
    if (threadIdx.x < 6) {
        long long v = s[threadIdx.x][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            const long long t = s[threadIdx.x][k];
            v = threadIdx.x < 3 ? (t < v ? t : v) : (t > v ? t : v);
        }
        part[6 * blockIdx.x + threadIdx.x] = v;
    }
}

// One block of 256 threads: each thread folds a stride of the block
// partials, then the warps and the block reduce; thread 0 sets the cube.
__global__ void __launch_bounds__(256) k_bbox_final(const long long* __restrict__ part, int nb, Geom* __restrict__ g)
{
    long long lo[3], hi[3];
    for (int a = 0; a < 3; ++a) lo[a] = 0x7fffffffffffffffLL, hi[a] = -lo[a] - 1;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const long long l = part[6 * b + a], h = part[6 * b + 3 + a];
            lo[a] = l < lo[a] ? l : lo[a];
            hi[a] = h > hi[a] ? h : hi[a];
        }
    __shared__ long long s[6][8];
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            const long long t0 = __shfl_xor_sync(kFull, lo[a], o), t1 = __shfl_xor_sync(kFull, hi[a], o);
            lo[a] = t0 < lo[a] ? t0 : lo[a];
            hi[a] = t1 > hi[a] ? t1 : hi[a];
        }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) s[a][w] = lo[a], s[3 + a][w] = hi[a];
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int a = 0; a < 3; ++a) {
        lo[a] = s[a][0], hi[a] = s[3 + a][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            lo[a] = s[a][k] < lo[a] ? s[a][k] : lo[a];
            hi[a] = s[3 + a][k] > hi[a] ? s[3 + a][k] : hi[a];
        }
    }
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) mn[a] = dval(lo[a]), mx[a] = dval(hi[a]);
    root_cube(mn, mx, g->lo, &g->S, &g->h);
    g->scale = ddiv(kGrid, g->S);
}

// ---- keys ---------------------------------------------------------------------

__global__ void k_keys(const double* __restrict__ pos, int64_t n, const Geom* __restrict__ g,
                       uint64_t* __restrict__ keys, uint32_t* __restrict__ vals)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t x = quantize(pos[3 * i], g->lo[0], g->scale);
    const uint32_t y = quantize(pos[3 * i + 1], g->lo[1], g->scale);
    const uint32_t z = quantize(pos[3 * i + 2], g->lo[2], g->scale);
    keys[i] = hilbert_key(x, y, z);
    vals[i] = (uint32_t)i;
}

// ---- stable LSD radix sort ----------------------------------------------------
// Block b counts the digits of its tile (hist, digit-major: hist[d * nblk +
// b]); an exclusive scan of hist gives each (digit, block) its output start.
// The scatter ranks each key after the keys of smaller digit in its tile and
// after the keys of equal digit that precede it (earlier warps of the block,
// earlier rounds and lower lanes of the warp), which keeps the sort stable;
// it stages the tile in that order in shared memory and then writes each
// digit's run of the tile to consecutive addresses from the run's global
// start (coalesced stores instead of one scattered store per key).

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                         int32_t* __restrict__ hist, int nblk)
{
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int k = 0; k < kRsItems; ++k) {
        const int64_t i = base + (int64_t)k * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & 255u)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

static_assert(kRsThreads == 256, "the scatter gives each of the 256 digits one thread");

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                            const uint32_t* __restrict__ vin, int64_t n, int shift,
                                                            const int32_t* __restrict__ offs, int nblk,
                                                            uint64_t* __restrict__ kout, uint32_t* __restrict__ vout)
{
    __shared__ int32_t wcount[kRsWarps][256];
    __shared__ int32_t dstart[256], gstart[256], wsum[kRsWarps];
    __shared__ uint64_t skey[kRsTile];
    __shared__ uint32_t sval[kRsTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int d = lane; d < 256; d += 32) wcount[w][d] = 0;
    __syncwarp();
    // warp w owns the contiguous run [base, base + 32 kRsItems) of the tile
    const int64_t b0 = (int64_t)blockIdx.x * kRsTile;
    const int64_t base = b0 + (int64_t)w * 32 * kRsItems;
    uint64_t key[kRsItems];
    uint32_t val[kRsItems];
    int dig[kRsItems];
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const int64_t i = base + r * 32 + lane;
        const bool ok = i < n;
        key[r] = ok ? kin[i] : 0;
        val[r] = ok ? vin[i] : 0;
        dig[r] = ok ? (int)((key[r] >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(kFull, dig[r]);
        if (ok && (peers & lt) == 0) wcount[w][dig[r]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // digit d = thread: exclusive prefix over the warps, the tile's count of
    // d, and (a block-wide scan over digits) the start of d's run in the tile
    {
        const int d = threadIdx.x;
        int32_t run = 0;
        for (int k = 0; k < kRsWarps; ++k) {
            const int32_t c = wcount[k][d];
            wcount[k][d] = run;
            run += c;
        }
        int32_t incl = run;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        int32_t excl = incl - run;
        for (int k = 0; k < w; ++k) excl += wsum[k];
        dstart[d] = excl;
        gstart[d] = offs[(int64_t)d * nblk + blockIdx.x];
        for (int k = 0; k < kRsWarps; ++k) wcount[k][d] += excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsItems; ++r) {
        const unsigned peers = __match_any_sync(kFull, dig[r]);
        const bool ok = dig[r] < 256;
        int32_t lp = 0;
        if (ok) lp = wcount[w][dig[r]] + __popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0) wcount[w][dig[r]] += __popc(peers);
        __syncwarp();
        if (ok) {
            skey[lp] = key[r];
            sval[lp] = val[r];
        }
    }
    __syncthreads();
    // the tile's valid keys fill [0, nvalid) of the staging in digit order
    const int nvalid = (int)(n - b0 < kRsTile ? n - b0 : kRsTile);
    for (int j = threadIdx.x; j < nvalid; j += kRsThreads) {
        const uint64_t k = skey[j];
        const int d = (int)((k >> shift) & 255u);
        const int64_t gp = (int64_t)gstart[d] + (j - dstart[d]);
        kout[gp] = k;
        vout[gp] = sval[j];
    }
}

// ---- tree order ------------------------------------------------------------------

__global__ void k_permute(const double* __restrict__ pos, const float* __restrict__ mass,
                          const uint32_t* __restrict__ order, int64_t n, const Geom* __restrict__ g,
                          otoo_src* __restrict__ src, int64_t* __restrict__ perm, int32_t* __restrict__ gq,
                          uint32_t* __restrict__ status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = order[k];
    if (i >= n) {  // the sort is a permutation; this only guards the reads
        atomicOr(status, kTreeBadSort);
        return;
    }
    otoo_src s;
    s.x = pos[3 * i];
    s.y = pos[3 * i + 1];
    s.z = pos[3 * i + 2];
    s.m = mass[i];
    s.pad = 0;
    src[k] = s;
    perm[k] = i;
    gq[3 * k] = (int32_t)quantize(s.x, g->lo[0], g->scale);
    gq[3 * k + 1] = (int32_t)quantize(s.y, g->lo[1], g->scale);
    gq[3 * k + 2] = (int32_t)quantize(s.z, g->lo[2], g->scale);
}

// ---- cells, one level at a time ---------------------------------------------------

struct Cells {
    int32_t* begin;
    int32_t* end;
    int32_t* level;
    int32_t* parent;
    int32_t* child0;
    int32_t* nchild;
};

// The levels' first cells live on the device (lev[L] = first cell of level
// L, lev[L + 1] = one past its last), so that a level is expanded without the
// host reading its size: each kernel reads the bounds and runs a grid-stride
// loop over 8 threads per cell (whole blocks per round, so that the
// 8-lane shuffles and the ballots see every lane).  stop != 0 (the cell
// capacity ran out) makes the rest of the expansion return at once.

// Thread (c, d): the start of the run of next-level digit >= d inside cell
// c = lo + t / 8 (a split cell's keys are sorted and share the cell's prefix,
// so its next digit does not decrease along the cell).  cnt[c - lo] = number
// of non-empty runs (children); starts go to dig[(c - lo) * 8 + d].
__global__ void k_expand_count(const int32_t* __restrict__ lev, int L, int leaf_size,
                               const uint64_t* __restrict__ keys, Cells c, int32_t* __restrict__ dig,
                               int32_t* __restrict__ cnt, const uint32_t* __restrict__ stop)
{
    if (*stop) return;
    const int32_t lo = lev[L], hi = lev[L + 1];
    const int64_t nt = 8 * (int64_t)(hi - lo);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nt; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const int32_t cell = lo + (int32_t)(t >> 3);
        const int d = (int)(t & 7);
        const bool in = t < nt;
        int32_t b = 0, e = 0;
        bool split = false;
        if (in) {
            b = c.begin[cell];
            e = c.end[cell];
            split = e - b > leaf_size && L < kLevels;
        }
        int32_t start = e;
        if (split) {
            const int shift = 3 * (kLevels - 1 - L);
            int32_t l = b, r = e;  // first index in [b, e) with digit >= d
            while (l < r) {
                const int32_t m = l + ((r - l) >> 1);
                if ((int)((keys[m] >> shift) & 7u) < d)
                    l = m + 1;
                else
                    r = m;
            }
            start = l;
        }
        // run d is [start_d, start_{d+1}), start_8 = e
        const int32_t next = __shfl_down_sync(kFull, start, 1, 8);
        const int32_t nxt = d == 7 ? e : next;
        const bool nonempty = split && start < nxt;
        const unsigned m = __ballot_sync(kFull, nonempty);
        if (in) {
            dig[(int64_t)(cell - lo) * 8 + d] = start;
            if (d == 0) cnt[cell - lo] = __popc((m >> (threadIdx.x & 24)) & 0xffu);
        }
    }
}

// Writes level L + 1: the children of level L's cells at lev[L + 1] +
// coff[c - lo] (coff: the exclusive scan of cnt, *total its sum), and
// lev[L + 2].  Children past cap are not written and set stop.
__global__ void k_expand_write(int32_t* __restrict__ lev, int L, Cells c, const int32_t* __restrict__ dig,
                               const int32_t* __restrict__ coff, const int64_t* __restrict__ total, int64_t cap,
                               uint32_t* __restrict__ stop)
{
    if (*stop) return;
    const int32_t lo = lev[L], hi = lev[L + 1];
    const int32_t next_base = hi;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t end = (int64_t)hi + *total;
        lev[L + 2] = (int32_t)(end < cap ? end : cap);
        if (end > cap) *stop = 1u;
    }
    const int64_t nt = 8 * (int64_t)(hi - lo);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nt; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + threadIdx.x;
        const int32_t cell = lo + (int32_t)(t >> 3);
        const int d = (int)(t & 7);
        const bool in = t < nt;
        int32_t start = 0, e = 0;
        if (in) {
            start = dig[(int64_t)(cell - lo) * 8 + d];
            e = c.end[cell];
        }
        const int32_t next = __shfl_down_sync(kFull, start, 1, 8);
        const int32_t nxt = d == 7 ? e : next;
        const bool nonempty = in && start < nxt;  // a cell that does not split has start = end for every digit
        const unsigned m = __ballot_sync(kFull, nonempty);
        const unsigned mine = (m >> (threadIdx.x & 24)) & 0xffu;
        if (!in) continue;
        const int32_t first = next_base + coff[cell - lo];
        if (d == 0) {
            c.child0[cell] = mine ? first : 0;
            c.nchild[cell] = __popc(mine);
        }
        if (nonempty) {
            const int64_t k = (int64_t)first + __popc(mine & ((1u << d) - 1u));
            if (k < cap) {
                c.begin[k] = start;
                c.end[k] = nxt;
                c.level[k] = L + 1;
                c.parent[k] = cell;
            }
        }
    }
}

// ---- moments ------------------------------------------------------------------------

struct Moments {
    double* m;      // [cap]
    double* com;    // [cap][3]
    double* q;      // [cap][6] central second moment Cxx Cyy Czz Cxy Cxz Cyz
    double* b2;     // [cap]
    unsigned long long* dmax2;  // [cap] bits of the largest squared distance (FP64), or of
                                //   the SPH radius (FP32, zero-extended)
};

// Cells [lo, hi), one thread each, in one pass over the cell's members
// (its particles for a leaf, its children for a parent): with x0 a member's
// position (a leaf's first particle, a parent's heaviest child's centre of
// mass) and d = x - x0, M = sum m, S1 = sum m d, S2 = sum m d d^T (+ the
// child's own central second moment C_c), then com = x0 + S1 / M and the
// central second moment C = S2 - S1 S1^T / M (the parallel-axis shift to the
// centre of mass).  S1 S1^T / M = M g g^T with g = com - x0, while C holds
// at least m_0 M / (M - m_0) g g^T (the reference member, mass m_0, against
// the rest), so the subtraction loses about log2((M - m_0) / m_0) bits: under
// 3 for a parent (the heaviest of up to 8 children), about log2 of the leaf
// size for equal masses in a leaf.  Stored: m, com, C (Cxx Cyy Czz Cxy Cxz
// Cyz) and B_2 = tr C; the records take the quadrupole Q = 3 C - tr(C) I.
// mode 1: leaves only; 2: parents only (their children done); else all.
__global__ void k_moments(int32_t lo, int32_t hi, const otoo_src* __restrict__ src, Cells c, Moments mo, int mode)
{
    const int32_t cell = lo + (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (cell >= hi) return;
    const int32_t nch = c.nchild[cell];
    if ((mode == 1 && nch != 0) || (mode == 2 && nch == 0)) return;
    double m = 0, s1[3] = {0, 0, 0}, s2[6] = {0, 0, 0, 0, 0, 0}, x0[3];
    if (nch == 0) {
        const int32_t b = c.begin[cell], e = c.end[cell];
        {
            const otoo_src p = src[b];
            x0[0] = p.x, x0[1] = p.y, x0[2] = p.z;
        }
#pragma unroll 1
        for (int32_t i = b; i < e; ++i) {
            const otoo_src p = src[i];
            const double mi = p.m;
            const double dx = p.x - x0[0], dy = p.y - x0[1], dz = p.z - x0[2];
            const double mx = mi * dx, my = mi * dy, mz = mi * dz;
            m += mi;
            s1[0] += mx, s1[1] += my, s1[2] += mz;
            s2[0] = fma(mx, dx, s2[0]), s2[1] = fma(my, dy, s2[1]), s2[2] = fma(mz, dz, s2[2]);
            s2[3] = fma(mx, dy, s2[3]), s2[4] = fma(mx, dz, s2[4]), s2[5] = fma(my, dz, s2[5]);
        }
    } else {
        const int32_t c0 = c.child0[cell];
        int32_t kh = c0;  // the heaviest child (positive doubles order like their bits)
        unsigned long long mh = 0;
        for (int32_t k = c0; k < c0 + nch; ++k) {
            const unsigned long long mb = (unsigned long long)__double_as_longlong(mo.m[k]);
            if (mb > mh) mh = mb, kh = k;
        }
        for (int a = 0; a < 3; ++a) x0[a] = mo.com[3 * kh + a];
#pragma unroll 1
        for (int32_t k = c0; k < c0 + nch; ++k) {
            const double mk = mo.m[k];
            const double dx = mo.com[3 * k] - x0[0], dy = mo.com[3 * k + 1] - x0[1], dz = mo.com[3 * k + 2] - x0[2];
            const double mx = mk * dx, my = mk * dy, mz = mk * dz;
            m += mk;
            s1[0] += mx, s1[1] += my, s1[2] += mz;
            s2[0] = fma(mx, dx, s2[0] + mo.q[6 * k]), s2[1] = fma(my, dy, s2[1] + mo.q[6 * k + 1]);
            s2[2] = fma(mz, dz, s2[2] + mo.q[6 * k + 2]), s2[3] = fma(mx, dy, s2[3] + mo.q[6 * k + 3]);
            s2[4] = fma(mx, dz, s2[4] + mo.q[6 * k + 4]), s2[5] = fma(my, dz, s2[5] + mo.q[6 * k + 5]);
        }
    }
    const double inv = 1.0 / m;
    const double gx = s1[0] * inv, gy = s1[1] * inv, gz = s1[2] * inv;  // com - x0
    mo.m[cell] = m;
    mo.com[3 * cell] = x0[0] + gx;
    mo.com[3 * cell + 1] = x0[1] + gy;
    mo.com[3 * cell + 2] = x0[2] + gz;
    const double cxx = fma(-s1[0], gx, s2[0]), cyy = fma(-s1[1], gy, s2[1]), czz = fma(-s1[2], gz, s2[2]);
    double* q = mo.q + 6 * (int64_t)cell;
    q[0] = cxx, q[1] = cyy, q[2] = czz;
    q[3] = fma(-s1[0], gy, s2[3]), q[4] = fma(-s1[0], gz, s2[4]), q[5] = fma(-s1[1], gz, s2[5]);
    mo.b2[cell] = cxx + cyy + czz;
    mo.dmax2[cell] = 0ull;
}

// FP32 distance |c~ - x~_j| between a cell's rounded centre of mass c~ and a
// rounded particle x~_j (k_bmax), and the particle's rounding bound
// e_j = 2^-23 (|x~| + |y~| + |z~|).
__device__ __forceinline__ float bmax_dist(const float4 cc, const float4 p, float& ej)
{
    const float dx = cc.x - p.x, dy = cc.y - p.y, dz = cc.z - p.z;
    ej = 0x1p-23f * (fabsf(p.x) + fabsf(p.y) + fabsf(p.z));
    return sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
}

// Work items, one warp each: warp w < n_cell takes the first kBmaxChunk
// particles of cell w; warp n_cell + k takes extra chunk k of the cells that
// hold more (extra_off: exclusive prefix over cells of their chunk counts
// minus one, so only those few warps search it).  The chunk's largest value
// goes to the cell by an atomic max on its bits (non-negative floating-point
// values order like their bit patterns).
//
// pk[j] = (x_j, y_j, z_j rounded to FP32, h_j or 0) in tree order,
// cf[cell] = (com rounded to FP32, e_c).  Rounding a value v to FP32 moves it
// by at most 2^-24 |v| per coordinate, so |com - x_j| lies within
// e_c + e_j (twice that bound, which also covers rounding in e itself) of
// |com~ - x~_j|, and the FP32 distance errs by a few 2^-24 relative, covered
// by a factor 1 -+ 2^-20.
//
// SPH (sph != 0): an upper bound on the cell's SPH radius, the largest
// |com - x_j| + h_j (Eq. SPH_RAD), in FP32 throughout; dmax2 holds the float
// bits, zero-extended.  The radius can only be larger than the exact one: a
// cell may keep particles that contribute W = 0 but never loses a neighbour.
//
// Absolute MAC: the largest squared distance in FP64, as the host computes
// it; dmax2 holds double bits.  A first FP32 pass finds a lower bound L on
// the chunk's largest distance; the FP64 distance is then taken only for the
// particles whose FP32 upper bound reaches L.  That set holds every particle
// whose FP64 value could be the largest (their exact distances lie within
// 2^-40 or so of the largest, far inside the bounds' margin), so the result
// is the same bits as the FP64 maximum over all particles.
__global__ void k_bmax(int64_t n_items, int32_t n_cell, const int32_t* __restrict__ extra_off,
                       const otoo_src* __restrict__ src, const float4* __restrict__ pk,
                       const float4* __restrict__ cf, Cells c, Moments mo, int sph)
{
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_items) return;
    int32_t cell;
    int64_t chunk;
    if (w < n_cell) {
        cell = (int32_t)w;
        chunk = 0;
    } else {
        const int64_t k = w - n_cell;
        int32_t l = 0, r = n_cell;  // last cell with extra_off <= k
        while (r - l > 1) {
            const int32_t m = l + ((r - l) >> 1);
            if (extra_off[m] <= k)
                l = m;
            else
                r = m;
        }
        cell = l;
        chunk = 1 + k - extra_off[cell];
    }
    const int32_t b = c.begin[cell], e = c.end[cell];
    const int64_t i0 = b + chunk * kBmaxChunk;
    const int64_t i1 = i0 + kBmaxChunk < e ? i0 + kBmaxChunk : e;
    const float4 cc = cf[cell];
    if (sph) {
        float vmax = 0.f;
        for (int64_t i = i0 + lane; i < i1; i += 32) {
            const float4 p = pk[i];
            float ej;
            const float d = bmax_dist(cc, p, ej);
            vmax = fmaxf(vmax, d + (p.w + ej));
        }
        for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(kFull, vmax, o));
        if (lane == 0)
            atomicMax(mo.dmax2 + cell, (unsigned long long)__float_as_uint((vmax + cc.w) * (1.0f + 0x1p-20f)));
        return;
    }
    float lo = 0.f;
    for (int64_t i = i0 + lane; i < i1; i += 32) {
        float ej;
        const float d = bmax_dist(cc, pk[i], ej);
        lo = fmaxf(lo, d * (1.0f - 0x1p-20f) - 2.0f * (ej + cc.w));
    }
    for (int o = 16; o > 0; o >>= 1) lo = fmaxf(lo, __shfl_xor_sync(kFull, lo, o));
    const double cx = mo.com[3 * cell], cy = mo.com[3 * cell + 1], cz = mo.com[3 * cell + 2];
    unsigned long long d2max = 0;
    for (int64_t i = i0 + lane; i < i1; i += 32) {
        float ej;
        const float d = bmax_dist(cc, pk[i], ej);
        if (!((d + 2.0f * (ej + cc.w)) * (1.0f + 0x1p-20f) < lo)) {  // NaN bounds count as candidates
            const otoo_src p = src[i];
            const double dx = cx - p.x, dy = cy - p.y, dz = cz - p.z;
            const unsigned long long v = (unsigned long long)__double_as_longlong(dx * dx + dy * dy + dz * dz);
            d2max = v > d2max ? v : d2max;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(kFull, d2max, o);
        d2max = v > d2max ? v : d2max;
    }
    if (lane == 0) atomicMax(mo.dmax2 + cell, d2max);
}

// Chunks of kBmaxChunk particles beyond the first, per cell, and the cell's
// FP32 centre of mass with its rounding bound e_c (k_bmax).
__global__ void k_chunks(int32_t n_cell, Cells c, const double* __restrict__ com, int32_t* __restrict__ extra,
                         float4* __restrict__ cf)
{
    const int32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= n_cell) return;
    const int32_t cnt = c.end[cell] - c.begin[cell];
    extra[cell] = (cnt + kBmaxChunk - 1) / kBmaxChunk - 1;
    const float x = (float)com[3 * cell], y = (float)com[3 * cell + 1], z = (float)com[3 * cell + 2];
    cf[cell] = make_float4(x, y, z, 0x1p-23f * (fabsf(x) + fabsf(y) + fabsf(z)));
}

// Tree-order FP32 positions with each particle's SPH radius, or 0 without h
// (k_bmax).
__global__ void k_bpack(int64_t n, const otoo_src* __restrict__ src, const float* __restrict__ h,
                        const int64_t* __restrict__ perm, float4* __restrict__ pk)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const otoo_src p = src[i];
    pk[i] = make_float4((float)p.x, (float)p.y, (float)p.z, h ? h[perm[i]] : 0.0f);
}

// ---- records and groups ----------------------------------------------------------

struct RecArgs {
    int64_t n_part;
    int32_t n_cell, use_quad, mac, n_crit;
    double delta, m_limit;
};

__global__ void k_records(RecArgs ra, const Geom* __restrict__ g, Cells c, Moments mo, const int32_t* __restrict__ gq,
                          otoo_src* __restrict__ src, otoo_quad* __restrict__ quad, otoo_wcell* __restrict__ wc,
                          otoo_wcell64* __restrict__ wc64, int32_t* __restrict__ level_out)
{
    const int32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ra.n_cell) return;
    const int L = c.level[cell];
    const int32_t b = c.begin[cell];
    const int sh = kLevels - L;
    const double side = cube_side(g->h, L);
    double lo[3], gc[3], com[3];
    for (int a = 0; a < 3; ++a) {
        const int64_t gcoord = gq[3 * (int64_t)b + a];
        const int64_t org = sh >= kLevels ? 0 : (gcoord >> sh) << sh;
        lo[a] = cube_lo(g->lo[a], org, g->h);
        gc[a] = cube_centre(lo[a], side);
        com[a] = mo.com[3 * cell + a];
    }
    const double m = mo.m[cell];
    otoo_src s;
    s.x = com[0];
    s.y = com[1];
    s.z = com[2];
    s.m = (float)m;
    s.pad = 0;
    src[ra.n_part + cell] = s;
    otoo_quad qd;
    const bool u = ra.use_quad != 0;
    // Q = 3 C - tr(C) I from the central second moment C
    const double* cm = mo.q + 6 * (int64_t)cell;
    const double tr = mo.b2[cell];
    qd.xx = u ? (float)(3.0 * cm[0] - tr) : 0.f;
    qd.yy = u ? (float)(3.0 * cm[1] - tr) : 0.f;
    qd.zz = u ? (float)(3.0 * cm[2] - tr) : 0.f;
    qd.xy = u ? (float)(3.0 * cm[3]) : 0.f;
    qd.xz = u ? (float)(3.0 * cm[4]) : 0.f;
    qd.yz = u ? (float)(3.0 * cm[5]) : 0.f;
    qd.b2 = u ? (float)tr : 0.f;
    qd.pad = 0.f;
    quad[cell] = qd;
    const double dm = __longlong_as_double((long long)mo.dmax2[cell]);
    const double rb = ra.mac == OTOO_MAC_SW    ? sw_radius(mo.b2[cell], __dsqrt_rn(dm), m, ra.delta, ra.m_limit, g->S)
                      : ra.mac == OTOO_MAC_SPH ? (double)__uint_as_float((unsigned)mo.dmax2[cell])
                                               : 0.0;
    otoo_wcell w;
    wcell_geometry(com, lo, gc, side, &w);
    w.nchild = c.nchild[cell];
    w.child0 = w.nchild > 0 ? c.child0[cell] : 0;
    w.begin = b;
    w.end = c.end[cell];
    w.rb = (float)rb;
    wc[cell] = w;
    otoo_wcell64 w64;
    for (int a = 0; a < 3; ++a) w64.lo[a] = lo[a], w64.com[a] = com[a], w64.gc[a] = gc[a];
    w64.side = side;
    w64.rb = rb;
    w64.pad = 0.0;
    wc64[cell] = w64;
    level_out[cell] = L;
}

// A group starts at the first particle of each maximal cell with at most
// n_crit particles, and every n_crit particles inside a leaf that holds more.
__global__ void k_group_flags(RecArgs ra, Cells c, int32_t* __restrict__ flag)
{
    const int32_t cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ra.n_cell) return;
    const int32_t b = c.begin[cell], e = c.end[cell], p = c.parent[cell];
    const int32_t cnt = e - b;
    const bool parent_big = p < 0 || c.end[p] - c.begin[p] > ra.n_crit;
    if (!parent_big) return;
    if (cnt <= ra.n_crit) {
        flag[b] = 1;
    } else if (c.nchild[cell] == 0) {
        for (int32_t k = b; k < e; k += ra.n_crit) flag[k] = 1;
    }
}

__global__ void k_group_write(int64_t n, const int32_t* __restrict__ flag, const int32_t* __restrict__ gidx,
                              int32_t* __restrict__ first)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n && flag[k]) first[gidx[k]] = (int32_t)k;
}

__global__ void k_group_count(int64_t n, int32_t G, const int32_t* __restrict__ first, int32_t* __restrict__ count)
{
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    count[g] = (g + 1 < G ? first[g + 1] : (int32_t)n) - first[g];
}

// ---- scans (exclusive, in place, int32) --------------------------------------------

constexpr int kScanThreads = 1024;

__device__ int64_t block_excl_scan64(int64_t v, int64_t* ws, int64_t* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int64_t w = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
        int64_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        ws[lane] = wi - w;
        if (lane == 31) ws[32] = wi;
    }
    __syncthreads();
    const int64_t r = ws[wid] + inc - v;
    *total = ws[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const int32_t* __restrict__ a, int64_t n,
                                                             int64_t* __restrict__ bsum)
{
    __shared__ int64_t ws[33];
    const int64_t i = (int64_t)blockIdx.x * kScanThreads + threadIdx.x;
    int64_t tot;
    block_excl_scan64(i < n ? a[i] : 0, ws, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(int64_t* __restrict__ bsum, int64_t nblk,
                                                            int64_t* __restrict__ total)
{
    __shared__ int64_t ws[33];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nblk; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        int64_t tot;
        const int64_t e = block_excl_scan64(i < nblk ? bsum[i] : 0, ws, &tot);
        if (i < nblk) bsum[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int32_t* __restrict__ a, int64_t n,
                                                              const int64_t* __restrict__ bsum)
{
    __shared__ int64_t ws[33];
    const int64_t i = (int64_t)blockIdx.x * kScanThreads + threadIdx.x;
    int64_t tot;
    const int64_t e = block_excl_scan64(i < n ? a[i] : 0, ws, &tot) + bsum[blockIdx.x];
    if (i < n) a[i] = (int32_t)e;
}

#define CUDA_TRY(expr)                                                                                 \
    do {                                                                                               \
        cudaError_t e_ = (expr);                                                                       \
        if (e_ != cudaSuccess) return set_error(OTOO_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));  \
    } while (0)

// exclusive scan of a[0, n) in place; the total to *total (device)
// The same three scans over a[0, n) with n = lev[L + 1] - lev[L] read on the
// device: grid-stride over blocks of kScanThreads (whole blocks per round).
__global__ void __launch_bounds__(kScanThreads) k_scan_sums_lev(const int32_t* __restrict__ a,
                                                                 const int32_t* __restrict__ lev, int L,
                                                                 int64_t* __restrict__ bsum)
{
    __shared__ int64_t ws[33];
    const int64_t n = lev[L + 1] - lev[L];
    for (int64_t blk = blockIdx.x; blk * kScanThreads < n; blk += gridDim.x) {
        const int64_t i = blk * kScanThreads + threadIdx.x;
        int64_t tot;
        block_excl_scan64(i < n ? a[i] : 0, ws, &tot);
        if (threadIdx.x == 0) bsum[blk] = tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top_lev(int64_t* __restrict__ bsum,
                                                                const int32_t* __restrict__ lev, int L,
                                                                int64_t* __restrict__ total)
{
    const int64_t n = lev[L + 1] - lev[L];
    const int64_t nblk = (n + kScanThreads - 1) / kScanThreads;
    __shared__ int64_t ws[33];
    int64_t carry = 0;
    for (int64_t b0 = 0; b0 < nblk; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        int64_t tot;
        const int64_t e = block_excl_scan64(i < nblk ? bsum[i] : 0, ws, &tot);
        if (i < nblk) bsum[i] = carry + e;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply_lev(int32_t* __restrict__ a,
                                                                  const int32_t* __restrict__ lev, int L,
                                                                  const int64_t* __restrict__ bsum)
{
    __shared__ int64_t ws[33];
    const int64_t n = lev[L + 1] - lev[L];
    for (int64_t blk = blockIdx.x; blk * kScanThreads < n; blk += gridDim.x) {
        const int64_t i = blk * kScanThreads + threadIdx.x;
        int64_t tot;
        const int64_t e = block_excl_scan64(i < n ? a[i] : 0, ws, &tot) + bsum[blk];
        if (i < n) a[i] = (int32_t)e;
    }
}

int scan32(int32_t* a, int64_t n, int64_t* bsum, int64_t* total, cudaStream_t s)
{
    const int64_t nblk = (n + kScanThreads - 1) / kScanThreads;
    if (nblk == 0) {
        CUDA_TRY(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
        return OTOO_OK;
    }
    k_scan_sums<<<(unsigned)nblk, kScanThreads, 0, s>>>(a, n, bsum);
    k_scan_top<<<1, kScanThreads, 0, s>>>(bsum, nblk, total);
    k_scan_apply<<<(unsigned)nblk, kScanThreads, 0, s>>>(a, n, bsum);
    CUDA_TRY(cudaGetLastError());
    return OTOO_OK;
}

// Scratch layout (byte offsets, each part 256-byte aligned).
struct Layout {
    size_t keys0, keys1, vals0, vals1, hist, bsum, part, geom, gq, cells[6], mom_m, mom_com, mom_q, mom_b2,
        mom_dmax, dig, cnt, flag, tot, lev, total;
};

size_t up(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(int64_t n, int64_t cap)
{
    Layout l;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += up(bytes);
        return at;
    };
    const int64_t nblk = (n + kRsTile - 1) / kRsTile;
    const int64_t big = n > cap ? n : cap;
    l.keys0 = take(8 * n);
    l.keys1 = take(8 * n);
    l.vals0 = take(4 * n);
    l.vals1 = take(4 * n);
    l.hist = take(4 * 256 * nblk);
    l.bsum = take(8 * ((256 * nblk + 8 * big) / kScanThreads + 8));
    l.part = take(8 * 6 * 1024);
    l.geom = take(sizeof(Geom));
    l.gq = take(12 * n);
    for (int k = 0; k < 6; ++k) l.cells[k] = take(4 * cap);
    l.mom_m = take(8 * cap);
    l.mom_com = take(24 * cap);
    l.mom_q = take(48 * cap);
    l.mom_b2 = take(8 * cap);
    l.mom_dmax = take(8 * cap);
    l.dig = take(32 * cap);
    l.cnt = take(4 * (big + 1));
    l.flag = take(4 * (n + 1));
    l.tot = take(64);
    l.lev = take(4 * (kLevels + 4) + 4);  // level bounds, then the stop word
    l.total = o;
    return l;
}

}  // namespace

extern "C" {

int64_t otoo_devtree_scratch_bytes(int64_t n_part, int64_t cap_cell)
{
    if (n_part < 1 || cap_cell < 1) return 0;
    return (int64_t)layout(n_part, cap_cell).total;
}

int otoo_devtree_build(const double* pos, const float* mass, otoo_devtree* t, void* scratch, int64_t scratch_bytes,
                       void* stream)
{
    otoo::Range range_("otoo_devtree_build");
    OTOO_REQUIRE(pos && mass && t && scratch, OTOO_EINVAL, "otoo_devtree_build: NULL pointer");
    const int64_t n = t->n_part, cap = t->cap_cell;
    OTOO_REQUIRE(n >= 1 && n <= INT32_MAX / 2 && cap >= 1 && n + cap <= INT32_MAX, OTOO_EINVAL,
                 "otoo_devtree_build: n_part / cap_cell out of range");
    OTOO_REQUIRE(t->leaf_size >= 1 && t->n_crit >= 1 && t->n_crit <= kMaxGroup, OTOO_EINVAL,
                 "otoo_devtree_build: leaf_size < 1 or n_crit outside [1, %d]", kMaxGroup);
    OTOO_REQUIRE(t->mac == OTOO_MAC_THETA || t->mac == OTOO_MAC_SW || t->mac == OTOO_MAC_SPH, OTOO_EINVAL,
                 "unknown mac %d", t->mac);
    OTOO_REQUIRE(t->mac != OTOO_MAC_SPH || t->h_sph, OTOO_EINVAL, "OTOO_MAC_SPH needs h_sph");
    OTOO_REQUIRE(t->mac != OTOO_MAC_SW || (t->delta >= 0.0 && std::isfinite(t->delta) && std::isfinite(t->m_limit)),
                 OTOO_EINVAL, "delta must be finite and >= 0, m_limit finite");
    OTOO_REQUIRE(t->src && t->quad && t->cell && t->cell64 && t->group_first && t->group_count && t->perm &&
                     t->cell_level && t->status,
                 OTOO_EINVAL, "otoo_devtree_build: NULL output array");
    const Layout ly = layout(n, cap);
    OTOO_REQUIRE(scratch_bytes >= (int64_t)ly.total, OTOO_EINVAL, "otoo_devtree_build: scratch too small (%lld < %lld)",
                 (long long)scratch_bytes, (long long)ly.total);
    OTOO_REQUIRE((reinterpret_cast<uintptr_t>(scratch) & 15) == 0, OTOO_EINVAL,
                 "otoo_devtree_build: scratch not 16-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char* base = static_cast<char*>(scratch);
    uint64_t* keys[2] = {reinterpret_cast<uint64_t*>(base + ly.keys0), reinterpret_cast<uint64_t*>(base + ly.keys1)};
    uint32_t* vals[2] = {reinterpret_cast<uint32_t*>(base + ly.vals0), reinterpret_cast<uint32_t*>(base + ly.vals1)};
    int32_t* hist = reinterpret_cast<int32_t*>(base + ly.hist);
    int64_t* bsum = reinterpret_cast<int64_t*>(base + ly.bsum);
    long long* part = reinterpret_cast<long long*>(base + ly.part);
    Geom* geom = reinterpret_cast<Geom*>(base + ly.geom);
    int32_t* gq = reinterpret_cast<int32_t*>(base + ly.gq);
    Cells c;
    c.begin = reinterpret_cast<int32_t*>(base + ly.cells[0]);
    c.end = reinterpret_cast<int32_t*>(base + ly.cells[1]);
    c.level = reinterpret_cast<int32_t*>(base + ly.cells[2]);
    c.parent = reinterpret_cast<int32_t*>(base + ly.cells[3]);
    c.child0 = reinterpret_cast<int32_t*>(base + ly.cells[4]);
    c.nchild = reinterpret_cast<int32_t*>(base + ly.cells[5]);
    Moments mo;
    mo.m = reinterpret_cast<double*>(base + ly.mom_m);
    mo.com = reinterpret_cast<double*>(base + ly.mom_com);
    mo.q = reinterpret_cast<double*>(base + ly.mom_q);
    mo.b2 = reinterpret_cast<double*>(base + ly.mom_b2);
    mo.dmax2 = reinterpret_cast<unsigned long long*>(base + ly.mom_dmax);
    int32_t* dig = reinterpret_cast<int32_t*>(base + ly.dig);
    int32_t* cnt = reinterpret_cast<int32_t*>(base + ly.cnt);
    int32_t* flag = reinterpret_cast<int32_t*>(base + ly.flag);
    int64_t* tot = reinterpret_cast<int64_t*>(base + ly.tot);
    uint32_t* status = t->status;

    // root cube, keys, sort
    CUDA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(uint32_t), s));
    const int nbb = (int)std::min<int64_t>(1024, (n + 255) / 256);
    k_bbox<<<nbb, 256, 0, s>>>(pos, mass, n, part, status);
    k_bbox_final<<<1, 256, 0, s>>>(part, nbb, geom);
    k_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, n, geom, keys[0], vals[0]);
    CUDA_TRY(cudaGetLastError());
    const int nblk = (int)((n + kRsTile - 1) / kRsTile);
    int cur = 0;
    for (int shift = 0; shift < 64; shift += 8) {
        k_rs_hist<<<nblk, kRsThreads, 0, s>>>(keys[cur], n, shift, hist, nblk);
        const int r = scan32(hist, (int64_t)256 * nblk, bsum, tot, s);
        if (r) return r;
        k_rs_scatter<<<nblk, kRsThreads, 0, s>>>(keys[cur], vals[cur], n, shift, hist, nblk, keys[cur ^ 1],
                                                 vals[cur ^ 1]);
        CUDA_TRY(cudaGetLastError());
        cur ^= 1;
    }
    k_permute<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, mass, vals[cur], n, geom, t->src, t->perm, gq,
                                                          status);
    CUDA_TRY(cudaGetLastError());
    uint32_t st = 0;
    CUDA_TRY(cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
    Geom hg;
    CUDA_TRY(cudaMemcpyAsync(&hg, geom, sizeof(hg), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (st & kTreeBadInput) return set_error(OTOO_EINVAL, "otoo_devtree_build: non-finite position or mass <= 0");
    if (st & kTreeBadSort) return set_error(OTOO_EDEVICE, "otoo_devtree_build: sort produced an invalid order");
    const uint64_t* skeys = keys[cur];

    // cells, level by level, the levels' bounds on the device (one read at
    // the end instead of one per level)
    const int32_t root[6] = {0, (int32_t)n, 0, -1, 0, 0};
    for (int k = 0; k < 6; ++k) {
        int32_t* arr = k == 0 ? c.begin : k == 1 ? c.end : k == 2 ? c.level : k == 3 ? c.parent : k == 4 ? c.child0 : c.nchild;
        CUDA_TRY(cudaMemcpyAsync(arr, &root[k], sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    int32_t* lev = reinterpret_cast<int32_t*>(base + ly.lev);
    uint32_t* stop = reinterpret_cast<uint32_t*>(lev + kLevels + 4);
    {
        static const int32_t lev01[2] = {0, 1};
        CUDA_TRY(cudaMemsetAsync(lev, 0, 4 * (kLevels + 4) + 4, s));
        CUDA_TRY(cudaMemcpyAsync(lev, lev01, sizeof(lev01), cudaMemcpyHostToDevice, s));
    }
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // grid-stride rounds: enough blocks to fill the GPU, no more than the
    // widest level could use (8 threads per cell, at most cap cells)
    const unsigned eg = (unsigned)std::min<int64_t>((int64_t)sms * 8, (8 * cap + 255) / 256);
    const unsigned sg = (unsigned)std::min<int64_t>((int64_t)sms * 2, (cap + kScanThreads - 1) / kScanThreads);
    for (int L = 0; L <= kLevels; ++L) {
        k_expand_count<<<eg, 256, 0, s>>>(lev, L, t->leaf_size, skeys, c, dig, cnt, stop);
        k_scan_sums_lev<<<sg, kScanThreads, 0, s>>>(cnt, lev, L, bsum);
        k_scan_top_lev<<<1, kScanThreads, 0, s>>>(bsum, lev, L, tot);
        k_scan_apply_lev<<<sg, kScanThreads, 0, s>>>(cnt, lev, L, bsum);
        k_expand_write<<<eg, 256, 0, s>>>(lev, L, c, dig, cnt, tot, cap, stop);
    }
    CUDA_TRY(cudaGetLastError());
    int32_t hlev[kLevels + 4];
    uint32_t hstop = 0;
    CUDA_TRY(cudaMemcpyAsync(hlev, lev, sizeof(hlev), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&hstop, stop, sizeof(hstop), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hstop) {
        t->n_cell = -1;
        return set_error(OTOO_ENOMEM, "otoo_devtree_build: more than cap_cell = %lld cells", (long long)cap);
    }
    // level L holds [hlev[L], hlev[L + 1]); the last non-empty level is the depth
    std::vector<int32_t> lev_lo(hlev, hlev + kLevels + 3);
    int depth = 0;
    for (int L = 0; L <= kLevels + 1; ++L)
        if (hlev[L + 1] > hlev[L]) depth = L;
    lev_lo.resize(depth + 2);
    const int32_t n_cell = lev_lo.back();

    // moments: every leaf in one launch, then the parents level by level,
    // deepest first
    k_moments<<<(unsigned)((n_cell + 127) / 128), 128, 0, s>>>(0, n_cell, t->src, c, mo, 1);
    for (int L = depth; L >= 0; --L) {
        const int32_t lo = lev_lo[L], hi = lev_lo[L + 1];
        if (hi > lo) k_moments<<<(unsigned)((hi - lo + 127) / 128), 128, 0, s>>>(lo, hi, t->src, c, mo, 2);
    }
    CUDA_TRY(cudaGetLastError());
    const bool sph = t->mac == OTOO_MAC_SPH;
    if (t->mac == OTOO_MAC_SW || sph) {
        // The sorted keys and the expansion digits are dead once the cells
        // exist: keys0..keys1 (two adjacent 256-byte-aligned parts of 8 n
        // bytes) hold the FP32 particles, dig (32 cap bytes) the FP32 centres.
        float4* pk = reinterpret_cast<float4*>(base + ly.keys0);
        float4* cf = reinterpret_cast<float4*>(dig);
        k_chunks<<<(unsigned)((n_cell + 255) / 256), 256, 0, s>>>(n_cell, c, mo.com, cnt, cf);
        k_bpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, t->src, sph ? t->h_sph : nullptr, t->perm, pk);
        const int r = scan32(cnt, n_cell, bsum, tot, s);
        if (r) return r;
        int64_t n_extra = 0;
        CUDA_TRY(cudaMemcpyAsync(&n_extra, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        const int64_t n_items = n_cell + n_extra;
        k_bmax<<<(unsigned)((n_items * 32 + 255) / 256), 256, 0, s>>>(n_items, n_cell, cnt, t->src, pk, cf, c, mo,
                                                                      sph ? 1 : 0);
        CUDA_TRY(cudaGetLastError());
    }
    RecArgs ra;
    ra.n_part = n;
    ra.n_cell = n_cell;
    ra.use_quad = t->use_quad ? 1 : 0;
    ra.mac = t->mac;
    ra.n_crit = t->n_crit;
    ra.delta = t->delta;
    ra.m_limit = t->m_limit;
    k_records<<<(unsigned)((n_cell + 127) / 128), 128, 0, s>>>(ra, geom, c, mo, gq, t->src, t->quad, t->cell,
                                                               t->cell64, t->cell_level);
    // groups
    CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t) * (size_t)n, s));
    k_group_flags<<<(unsigned)((n_cell + 255) / 256), 256, 0, s>>>(ra, c, flag);
    CUDA_TRY(cudaMemcpyAsync(cnt, flag, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    const int r = scan32(cnt, n, bsum, tot, s);
    if (r) return r;
    k_group_write<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, flag, cnt, t->group_first);
    int64_t G = 0;
    CUDA_TRY(cudaMemcpyAsync(&G, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    k_group_count<<<(unsigned)((G + 255) / 256), 256, 0, s>>>(n, (int32_t)G, t->group_first, t->group_count);
    CUDA_TRY(cudaGetLastError());
    t->n_cell = n_cell;
    t->n_groups = G;
    t->depth = depth;
    for (int a = 0; a < 3; ++a) t->root_lo[a] = hg.lo[a];
    t->root_side = hg.S;
    return OTOO_OK;
}

}  // extern "C"
