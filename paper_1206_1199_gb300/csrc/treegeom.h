// Tree geometry shared by the host build (tree.cpp) and the device build
// (tree_build.cu): the root cube, the 2^21 grid, the Hilbert key, the cube of
// a cell, the absolute MAC's radius and the FP32 walk record of a cell.
// Every FP64 operation is explicitly rounded (no contraction on either
// side), so both builds compute the same bits.
#pragma once
#include <stdint.h>

#include <cmath>

#include "otoo.h"

#ifdef __CUDACC__
#define OTOO_HD __host__ __device__ __forceinline__
#else
#define OTOO_HD inline
#endif

namespace otoo {

constexpr int kLevels = 21;                 // 2^21 grid cells per axis, 63-bit keys
constexpr double kGrid = 2097152.0;         // 2^21

OTOO_HD double dadd(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
OTOO_HD double dsub(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}
OTOO_HD double dmul(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
OTOO_HD double ddiv(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __ddiv_rn(a, b);
#else
    return a / b;
#endif
}
OTOO_HD double dsqrt(double a)
{
#ifdef __CUDA_ARCH__
    return __dsqrt_rn(a);
#else
    return std::sqrt(a);
#endif
}

// Root cube (Section III-B, step 1): centred on the bounding box [mn, mx],
// side = largest extent * (1 + 1e-12) (1 when all points coincide); h = side
// of one grid step.
OTOO_HD void root_cube(const double mn[3], const double mx[3], double lo[3], double* S, double* h)
{
    double ext = 0;
    for (int a = 0; a < 3; ++a) {
        const double e = dsub(mx[a], mn[a]);
        if (e > ext) ext = e;
    }
    double s = dmul(ext, 1.0 + 1e-12);
    if (!(s > 0.0)) s = 1.0;
    for (int a = 0; a < 3; ++a) lo[a] = dsub(dmul(dadd(mn[a], mx[a]), 0.5), dmul(0.5, s));
    *S = s;
    *h = ddiv(s, kGrid);
}

// Grid coordinate of x on an axis (Section III-B, step 2), clamped.
OTOO_HD uint32_t quantize(double x, double lo, double scale)
{
    double q = floor(dmul(dsub(x, lo), scale));
    if (q < 0.0) q = 0.0;
    if (q > kGrid - 1.0) q = kGrid - 1.0;
    return (uint32_t)q;
}

// Hilbert index of a point on the 2^21 grid: Skilling's transpose method
// (J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004):
// undo the excess rotations/reflections level by level, Gray-encode, then
// interleave the transposed bits from the top level down.  The top 3L bits
// name the level-L cube that holds the point, so a sort by key keeps every
// cell contiguous (the property the paper's Morton-to-Hilbert step keeps).
OTOO_HD uint64_t hilbert_key(uint32_t x0, uint32_t x1, uint32_t x2)
{
    uint32_t X[3] = {x0, x1, x2};
    const uint32_t M = 1u << (kLevels - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    uint64_t key = 0;
    for (int b = kLevels - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

// Cube of a cell at `level` whose integer origin on the grid is org:
// side = h 2^(21 - level), lower corner = lo + org h, centre = corner + side/2.
OTOO_HD double cube_side(double h, int level) { return dmul(h, (double)((int64_t)1 << (kLevels - level))); }
OTOO_HD double cube_lo(double root_lo, int64_t org, double h) { return dadd(root_lo, dmul((double)org, h)); }
OTOO_HD double cube_centre(double lo, double side) { return dadd(lo, dmul(0.5, side)); }

// Bounding radius of the absolute MAC (Eq. SW_MAC): where the monopole error
// bound 3 B_2 / (d^2 (d - b_max)^2) equals delta; 2 S_root for cells heavier
// than m_limit (never accepted, Section III-C); infinite for delta = 0.
OTOO_HD double sw_radius(double b2, double bmax, double m, double delta, double m_limit, double s_root)
{
    if (m_limit > 0.0 && m > m_limit) return dmul(2.0, s_root);
    if (!(delta > 0.0)) return HUGE_VAL;
    const double hb = dmul(0.5, bmax);
    return dadd(hb, dsqrt(dadd(dmul(hb, hb), dsqrt(ddiv(dmul(3.0, b2), delta)))));
}

// FP32 data of a cell's walk record (otoo_wcell) from its FP64 geometry:
// centre of mass as a float pair, its offset from the cube's lower corner,
// the side, and s = |com - cube centre| computed in FP64 then rounded.
OTOO_HD void wcell_geometry(const double com[3], const double lo[3], const double gc[3], double side,
                            otoo_wcell* w)
{
    double s2 = 0;
    for (int a = 0; a < 3; ++a) {
        w->com_hi[a] = (float)com[a];
        w->com_lo[a] = (float)dsub(com[a], (double)w->com_hi[a]);
        w->e[a] = (float)dsub(com[a], lo[a]);
        const double e = dsub(com[a], gc[a]);
        s2 = dadd(s2, dmul(e, e));
    }
    w->side = (float)side;
    w->s = (float)dsqrt(s2);
}

}  // namespace otoo
