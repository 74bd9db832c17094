// FP32 force kernel with packed two-wide FP32 arithmetic (included by
// force.cu after force_warp.cuh).
//
// The same work decomposition as k_force_warp (one work item per warp, IB
// targets per lane, lane subsets interleaved over the staged entries), but a
// lane evaluates two consecutive list entries at once: the shared-memory tile
// holds "pair records" whose fields are (entry 2m, entry 2m+1) float pairs,
// and every FP32 operation of the pair law is a packed fma/mul/add.f32x2
// (PTX) acting on both entries.  A packed instruction issues once for two
// FP32 operations, so the FP32 pipe rather than instruction issue bounds the
// kernel.  The reciprocal square root stays two scalar MUFU operations.
//
// Pair records: a cell tile stores 80 bytes per pair (x | y | z | m | -Qxx |
// -Qyy | B_2 eps^2 | -Qxy | -Qxz | -Qyz, each two floats; -Qzz is rebuilt
// from the traceless diagonal); a particle tile 32 bytes (x | y | z | m).
// Each field loads straight into a packed operand.  The quadrupole is stored
// negated so that the law needs no negation: with n = -Q r and u = r.n +
// B_2 eps^2, phi -= m q - (1/2) u q^5, a += (m q^3 - (5/2) u q^7) r + q^5 n.
// The potential is accumulated as a positive sum and negated at the end.
// The packed arithmetic (f2 operations, pair_mono2, pair_quad2, the record
// layout and the evaluation loops) is in pair.cuh.

// Packed operands take register pairs: fewer resident warps than the scalar
// kernel, each with twice the independent FP32 work per instruction.
#ifndef OTOO_W2_WARPS
#define OTOO_W2_WARPS 16  // resident warps per SM asked for at IB >= 2
#endif
#ifndef OTOO_W2_QUNROLL
#define OTOO_W2_QUNROLL 3  // pair records per step of the cell loop (3: 45.4 ms, 2: 46.0, 4: 45.5 at N = 2^23)
#endif
#ifndef OTOO_W2_MUNROLL
#define OTOO_W2_MUNROLL 3  // pair records per step of the particle loop (3: 45.1 ms, 2: 45.3, 4: 45.6)
#endif
constexpr int warp2_min_blocks(int nw, int ib) { return (ib == 1 ? 20 : OTOO_W2_WARPS) / nw; }

template <int NW, int IB, int SPL>
__global__ void __launch_bounds__(NW * 32, warp2_min_blocks(NW, IB)) k_force_warp2(const otoo_dev_system sys,
                                                                                  double* __restrict__ accel,
                                                                                  double* __restrict__ pot)
{
    constexpr int T = 32 * SPL;          // entries per tile at most
    constexpr int TP = T / 2;            // pair records per tile at most
    constexpr int PPL = (TP + 31) / 32;  // pair records staged per lane
    __shared__ float4 s_rec[NW][kCellRecF4 * TP];

    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint32_t* status = sys.counter + 1;
    const float4* __restrict__ ff = reinterpret_cast<const float4*>(sys.split);
    const bool has_quad = sys.quad != nullptr;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const f2 zero2 = f2pack(0.f, 0.f);

    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(sys.counter, 1u);
        it = __shfl_sync(kFull, it, 0);
        if (it >= sys.n_items) break;

        const otoo_item item = sys.items[it];
        otoo_group grp;
        if (!item_ok(sys, item, grp, 32 * IB)) {
            if (lane == 0) atomicOr(status, kBadItem);
            continue;
        }

        const int ni = item.ni;
        const int P = (ni + IB - 1) / IB;
        const int nsub = 32 / P;
        const int islot = lane % P, js = lane / P;
        const bool active = js < nsub;
        // pair records per tile: a multiple of nsub (a tile with fewer records
        // than nsub holds nsub, some of them zero)
        const int TEP = TP >= nsub ? (TP / nsub) * nsub : nsub;
        const int TE = 2 * TEP;  // entries per tile
        const float eps2 = (float)grp.eps2;
        const f2 e2 = f2pack(eps2, eps2);
        const float cx = __double2float_rn(grp.cx), cy = __double2float_rn(grp.cy), cz = __double2float_rn(grp.cz);

        f2 nx[IB], ny[IB], nz[IB];
        Acc<float> acc[IB];
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            const int i = islot + k * P;
            float x = 0.f, y = 0.f, z = 0.f;
            if (active && i < ni) {
                const int64_t t = (int64_t)grp.first + item.i0 + i;
                const float4 h = __ldg(ff + 2 * t);
                const float4 l = __ldg(ff + 2 * t + 1);
                x = rel32(h.x, l.x, cx);
                y = rel32(h.y, l.y, cy);
                z = rel32(h.z, l.z, cz);
            }
            nx[k] = f2pack(-x, -x);
            ny[k] = f2pack(-y, -y);
            nz[k] = f2pack(-z, -z);
            acc[k].zero();
        }

        const int c0 = item.j0, c1 = min(item.j1, grp.n_cell);
        const int p0 = max(item.j0, grp.n_cell), p1 = item.j1;
        const int ntc = c1 > c0 ? (c1 - c0 + TE - 1) / TE : 0;
        const int ntp = p1 > p0 ? (p1 - p0 + TE - 1) / TE : 0;
        const int nt = ntc + ntp;
        const int32_t* __restrict__ lst = sys.list + grp.list_off;
        float4* __restrict__ rec = s_rec[wid];

        // list indices of the next tile (entries 2m, 2m+1 of this lane's pairs)
        int nidx[PPL][2];
        auto load_idx = [&](int t) {
            const bool cell = t < ntc;
            const int base = cell ? c0 + t * TE : p0 + (t - ntc) * TE;
            const int cnt = cell ? min(TE, c1 - base) : min(TE, p1 - base);
#pragma unroll
            for (int pp = 0; pp < PPL; ++pp)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * (lane + 32 * pp) + h;
                    nidx[pp][h] = k < cnt ? __ldg(lst + base + k) : 0;
                }
        };
        if (nt > 0) load_idx(0);

        for (int t = 0; t < nt; ++t) {
            const bool cell = t < ntc;
            const bool cq = cell && has_quad;
            const int base = cell ? c0 + t * TE : p0 + (t - ntc) * TE;
            const int cnt = cell ? min(TE, c1 - base) : min(TE, p1 - base);
            const int npair = (cnt + 1) / 2;
            const int npair_pad = (npair + nsub - 1) / nsub * nsub;

            // stage this lane's pair records: loads of both entries first
#pragma unroll
            for (int pp = 0; pp < PPL; ++pp) {
                const int m = lane + 32 * pp;
                if (m >= npair_pad) continue;
                float4 hh[2], ll[2], qa[2], qb[2];
                bool real[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * m + h;
                    real[h] = k < cnt;
                    hh[h] = ll[h] = qa[h] = qb[h] = zero4;
                    if (real[h]) {
                        const int idx = nidx[pp][h];
                        const bool good =
                            cell ? (idx >= sys.n_part && idx < sys.n_src) : (idx >= 0 && idx < sys.n_part);
                        if (good) {
                            // a source's float pair and a cell's quadrupole: one 32-byte load each
                            ld256x2(ff + 2 * (int64_t)idx, hh[h], ll[h]);
                            if (cq) ld256x2(reinterpret_cast<const float4*>(sys.quad + (idx - sys.n_part)), qa[h], qb[h]);
                        } else {
                            atomicOr(status, kBadIndex);
                            real[h] = false;
                        }
                    }
                }
                float x[2], y[2], z[2], w[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // padding and rejected entries loaded as zeros: mass (and
                    // quadrupole) 0, so they add exactly nothing
                    x[h] = rel32(hh[h].x, ll[h].x, cx);
                    y[h] = rel32(hh[h].y, ll[h].y, cy);
                    z[h] = rel32(hh[h].z, ll[h].z, cz);
                    w[h] = hh[h].w;
                }
                put_rec2(rec, m, cq, x, y, z, w, qa, qb, eps2);
            }
            if (t + 1 < nt) load_idx(t + 1);
            __syncwarp();

            if (active) {
                Acc2 P2[IB];
#pragma unroll
                for (int k = 0; k < IB; ++k) P2[k].v[0] = P2[k].v[1] = P2[k].v[2] = P2[k].v[3] = zero2;
                const int niter = npair_pad / nsub;
                if (cq)
                    eval_cells2<IB, OTOO_W2_QUNROLL>(rec, js, nsub, niter, nx, ny, nz, e2, P2);
                else
                    eval_parts2<IB, OTOO_W2_MUNROLL>(rec, js, nsub, niter, nx, ny, nz, e2, P2);
#pragma unroll
                for (int k = 0; k < IB; ++k) {
                    float s[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float lo, hi;
                        f2unpack(P2[k].v[c], lo, hi);
                        s[c] = lo + hi;
                    }
                    acc[k].add(s);
                }
            }
            __syncwarp();
        }

        // merge the lane subsets into the js == 0 lanes (pairwise, in a fixed
        // order) with a compensated FP32 sum; one conversion to FP64 per output
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            double a[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float S = acc[k].s[c], C = acc[k].c[c];
                merge_subsets(S, C, js, nsub, P);
                a[c] = (double)S - (double)C;
            }
            a[3] = -a[3];
            const int i = islot + k * P;
            if (js == 0 && i < ni) {
                if (item.j0 == 0) {
                    // the self pair added exactly -m_i rsqrt(eps^2) in FP32: take the same value out
                    const float4 h = __ldg(ff + 2 * ((int64_t)grp.first + item.i0 + i));
                    a[3] += (double)(h.w * rsqrt_r(eps2));
                }
                write_target(sys, grp, item, i, a, accel, pot);
            }
        }
    }
}
