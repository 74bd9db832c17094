// FP32 and FP64 pair arithmetic of the force step, shared by the list-driven
// force kernels (force.cu) and the walk fused with the force (walk.cu):
// Plummer-softened particle / monopole pairs and quadrupole cell pairs
// (Section II: a cell acts as a virtual particle at its centre of mass; the
// quadrupole term is this library's extension), scalar and packed two-wide
// FP32 forms, compensated running sums and the merge of a warp's lane
// subsets.  Included inside each translation unit's anonymous namespace.
#pragma once

template <typename R> struct V4;
template <> struct __align__(16) V4<float> { float x, y, z, w; };
template <> struct __align__(32) V4<double> { double x, y, z, w; };
template <typename R> struct V2;
template <> struct __align__(8) V2<float> { float x, y; };
template <> struct __align__(16) V2<double> { double x, y; };

// FP32 reciprocal square root: the hardware approximation (PTX
// rsqrt.approx.ftz.f32, relative error about 2^-23); the argument r^2 + eps^2
// is never subnormal for eps > 0, so flushing subnormals changes nothing.
__device__ __forceinline__ float rsqrt_r(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double rsqrt_r(double x) { return rsqrt(x); }

// Centre-relative FP32 coordinate of the FP32 form: (hi - c) + lo, with
// (hi, lo) the float pair of an FP64 coordinate (hi = x rounded to FP32, lo
// = (x - hi) rounded) and c the group centre rounded to FP32.  hi - c is
// exact whenever hi is within a factor of two of c (Sterbenz), so near
// entries get the FP64 difference rounded once (up to the rounding of lo,
// 2^-25 of an FP32 ulp of x); far entries are within about one FP32 ulp.
__device__ __forceinline__ float rel32(float hi, float lo, float c) { return __fadd_rn(__fsub_rn(hi, c), lo); }

constexpr unsigned kFull = 0xffffffffu;

// Running sum of one target particle: FP32 with Kahan compensation c (the sum
// is s - c), FP64 plain.
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
template <> __device__ __forceinline__ double Acc<float>::value(int k) const { return (double)s[k] - (double)c[k]; }
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

// Quadrupole cell: the second-order Taylor term of the softened pair law
// about the cell's centre of mass.  With q = (r^2 + eps^2)^(-1/2), the
// traceless Q and w = r.Q.r - B_2 eps^2 (B_2 = sum m |x - com|^2; the B_2
// part vanishes without softening):
//   phi -= m q + (1/2) w q^5,  a += (m q^3 + (5/2) w q^7) r - q^5 Q r.
// qa = (Qxx, Qyy, Qzz, Qxy), qb = (Qxz, Qyz, B_2 eps^2, -).
template <typename R>
__device__ __forceinline__ void pair_quad(const V4<R>& s, const V4<R>& qa, const V4<R>& qb, R xi, R yi, R zi,
                                          R eps2, R p[4])
{
    const R rx = s.x - xi, ry = s.y - yi, rz = s.z - zi;
    const R r2 = fma(rx, rx, fma(ry, ry, fma(rz, rz, eps2)));
    const R q = rsqrt_r(r2);
    const R q2 = q * q;
    const R mq = s.w * q;
    const R qr0 = fma(qa.x, rx, fma(qa.w, ry, qb.x * rz));
    const R qr1 = fma(qa.w, rx, fma(qa.y, ry, qb.y * rz));
    const R qr2 = fma(qb.x, rx, fma(qb.y, ry, qa.z * rz));
    const R w = fma(rx, qr0, fma(ry, qr1, fma(rz, qr2, -qb.z)));
    const R q5 = q * (q2 * q2);
    const R t = w * q5;
    p[3] -= fma(R(0.5), t, mq);
    // radial coefficient m q^3 + (5/2) w q^7 = q^2 (m q + (5/2) w q^5)
    const R cr = q2 * fma(R(2.5), t, mq);
    p[0] = fma(cr, rx, fma(-q5, qr0, p[0]));
    p[1] = fma(cr, ry, fma(-q5, qr1, p[1]));
    p[2] = fma(cr, rz, fma(-q5, qr2, p[2]));
}

typedef unsigned long long f2;

__device__ __forceinline__ f2 f2pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2unpack(f2 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 f2add(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2sub(f2 a, f2 b)
{
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2mul(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2fma(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2rsqrt(f2 a)
{
    float lo, hi;
    f2unpack(a, lo, hi);
    return f2pack(rsqrt_r(lo), rsqrt_r(hi));
}

// Accumulator of one target over packed entry pairs: A[0..2] acceleration,
// A[3] the positive potential sum (the potential with the opposite sign).
struct Acc2 {
    f2 v[4];
};

// Two particle entries (or monopole cells) against one target; nx = -x_i
// broadcast:  A[3] += m q,  A[0..2] += m q^3 r.
__device__ __forceinline__ void pair_mono2(f2 sx, f2 sy, f2 sz, f2 m, f2 nx, f2 ny, f2 nz, f2 e2, Acc2& A)
{
    const f2 rx = f2add(sx, nx), ry = f2add(sy, ny), rz = f2add(sz, nz);
    const f2 r2 = f2fma(rx, rx, f2fma(ry, ry, f2fma(rz, rz, e2)));
    const f2 q = f2rsqrt(r2);
    const f2 mq = f2mul(m, q);
    const f2 mq3 = f2mul(mq, f2mul(q, q));
    A.v[3] = f2add(A.v[3], mq);
    A.v[0] = f2fma(mq3, rx, A.v[0]);
    A.v[1] = f2fma(mq3, ry, A.v[1]);
    A.v[2] = f2fma(mq3, rz, A.v[2]);
}

// Two quadrupole cells against one target: the law of pair_quad with the
// fields of -Q, n = -Q r and u = r.n + B_2 eps^2 = -w (te = B_2 eps^2):
//   A[3] += m q - (1/2) u q^5,  A[0..2] += (m q^3 - (5/2) u q^7) r + q^5 n;
// mhalf = (-1/2, -1/2), m5half = (-5/2, -5/2).
__device__ __forceinline__ void pair_quad2(f2 sx, f2 sy, f2 sz, f2 m, f2 nqxx, f2 nqyy, f2 nqzz, f2 nqxy, f2 nqxz,
                                           f2 nqyz, f2 te, f2 nx, f2 ny, f2 nz, f2 e2, f2 mhalf, f2 m5half, Acc2& A)
{
    const f2 rx = f2add(sx, nx), ry = f2add(sy, ny), rz = f2add(sz, nz);
    const f2 r2 = f2fma(rx, rx, f2fma(ry, ry, f2fma(rz, rz, e2)));
    const f2 q = f2rsqrt(r2);
    const f2 q2 = f2mul(q, q);
    const f2 mq = f2mul(m, q);
    const f2 n0 = f2fma(nqxx, rx, f2fma(nqxy, ry, f2mul(nqxz, rz)));
    const f2 n1 = f2fma(nqxy, rx, f2fma(nqyy, ry, f2mul(nqyz, rz)));
    const f2 n2 = f2fma(nqxz, rx, f2fma(nqyz, ry, f2mul(nqzz, rz)));
    const f2 u = f2fma(rx, n0, f2fma(ry, n1, f2fma(rz, n2, te)));
    const f2 q5 = f2mul(q, f2mul(q2, q2));
    const f2 tu = f2mul(u, q5);
    A.v[3] = f2add(A.v[3], f2fma(mhalf, tu, mq));
    // radial coefficient m q^3 - (5/2) u q^7 = q^2 (m q - (5/2) u q^5)
    const f2 cr = f2mul(q2, f2fma(m5half, tu, mq));
    A.v[0] = f2fma(cr, rx, f2fma(q5, n0, A.v[0]));
    A.v[1] = f2fma(cr, ry, f2fma(q5, n1, A.v[1]));
    A.v[2] = f2fma(cr, rz, f2fma(q5, n2, A.v[2]));
}

// Pair records of the packed kernels (k_force_warp2 and the walk fused with
// the force): two consecutive entries of a tile, each field a float pair
// (entry 2m, entry 2m + 1) so that it loads straight into the 64-bit
// operand of a packed instruction.  A particle record holds x | y | z | m
// (32 bytes); a cell record x | y | z | m | -Qxx | -Qyy | B_2 eps^2 | -Qxy |
// -Qxz | -Qyz (80 bytes): -Qzz = Qxx + Qyy is rebuilt from the other two
// diagonal terms (Q is traceless) by two packed subtractions per record,
// which measured faster than a sixth 16-byte slot per record (and storing
// -m with Q itself, which saves five negations per staged cell, measured 1%
// slower).  Coordinates are relative to the group centre.
constexpr int kPartRecF4 = 2;  // 16-byte slots per particle record
constexpr int kCellRecF4 = 5;  // 16-byte slots per cell record

// Writes pair record m of a tile from the two entries' centre-relative
// positions x, y, z, masses w and (cells) quadrupoles qa = (xx, yy, zz, xy),
// qb = (xz, yz, B_2, -), with e2 the group's softening^2.
__device__ __forceinline__ void put_rec2(float4* rec, int m, bool cellq, const float x[2], const float y[2],
                                         const float z[2], const float w[2], const float4 qa[2], const float4 qb[2],
                                         float e2)
{
    if (cellq) {
        float4* r = rec + kCellRecF4 * m;
        r[0] = make_float4(x[0], x[1], y[0], y[1]);
        r[1] = make_float4(z[0], z[1], w[0], w[1]);
        r[2] = make_float4(-qa[0].x, -qa[1].x, -qa[0].y, -qa[1].y);
        r[3] = make_float4(qb[0].z * e2, qb[1].z * e2, -qa[0].w, -qa[1].w);
        r[4] = make_float4(-qb[0].x, -qb[1].x, -qb[0].y, -qb[1].y);
    } else {
        float4* r = rec + kPartRecF4 * m;
        r[0] = make_float4(x[0], x[1], y[0], y[1]);
        r[1] = make_float4(z[0], z[1], w[0], w[1]);
    }
}

// Evaluates niter pair records per lane subset (records js, js + nsub, ...)
// against the lane's IB targets (nx, ny, nz = minus the target's
// centre-relative coordinates, as float pairs), accumulating into P2.
template <int IB, int UNROLL>
__device__ __forceinline__ void eval_cells2(const float4* rec, int js, int nsub, int niter, const f2 nx[IB],
                                            const f2 ny[IB], const f2 nz[IB], f2 e2, Acc2 P2[IB])
{
    const f2 mhalf = f2pack(-0.5f, -0.5f), m5half = f2pack(-2.5f, -2.5f), zero2 = f2pack(0.f, 0.f);
    const ulonglong2* __restrict__ r = reinterpret_cast<const ulonglong2*>(rec) + kCellRecF4 * js;
    const int S = kCellRecF4 * nsub;
#pragma unroll UNROLL
    for (int n = 0; n < niter; ++n, r += S) {
        const ulonglong2 a = r[0], b = r[1], c = r[2], d = r[3], e = r[4];
        const f2 nqzz = f2sub(f2sub(zero2, c.x), c.y);
#pragma unroll
        for (int k = 0; k < IB; ++k)
            pair_quad2(a.x, a.y, b.x, b.y, c.x, c.y, nqzz, d.y, e.x, e.y, d.x, nx[k], ny[k], nz[k], e2, mhalf, m5half,
                       P2[k]);
    }
}

template <int IB, int UNROLL>
__device__ __forceinline__ void eval_parts2(const float4* rec, int js, int nsub, int niter, const f2 nx[IB],
                                            const f2 ny[IB], const f2 nz[IB], f2 e2, Acc2 P2[IB])
{
    const ulonglong2* __restrict__ r = reinterpret_cast<const ulonglong2*>(rec) + kPartRecF4 * js;
    const int S = kPartRecF4 * nsub;
#pragma unroll UNROLL
    for (int n = 0; n < niter; ++n, r += S) {
        const ulonglong2 a = r[0], b = r[1];
#pragma unroll
        for (int k = 0; k < IB; ++k) pair_mono2(a.x, a.y, b.x, b.y, nx[k], ny[k], nz[k], e2, P2[k]);
    }
}

// Merges the compensated sums (S, C) of a warp's nsub lane subsets into the
// js == 0 lanes: subset js + d is added into subset js for d = 1, 2, 4, ...
// while js is a multiple of 2d (a fixed pairwise order, so the result does not
// depend on timing).  Lane islot + js * P holds subset js of target slot
// islot; every lane of the warp takes part in the shuffles.
__device__ __forceinline__ void merge_subsets(float& S, float& C, int js, int nsub, int P)
{
    for (int d = 1; d < nsub; d *= 2) {
        const float so = __shfl_down_sync(kFull, S, d * P);
        const float co = __shfl_down_sync(kFull, C, d * P);
        if ((js & (2 * d - 1)) == 0 && js + d < nsub) {
            const float y = __fsub_rn(__fsub_rn(so, co), C);
            const float tt = __fadd_rn(S, y);
            C = __fsub_rn(__fsub_rn(tt, S), y);
            S = tt;
        }
    }
}


// One 32-byte sector per load (256-bit vector load, sm_100 and later): the
// two consecutive float4 at p (32-byte aligned) in one request.
__device__ __forceinline__ void ld256x2(const float4* p, float4& a, float4& b)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}
