// FP32 force kernel, one work item per warp (included by force.cu, inside its
// anonymous namespace, after the pair laws and the item helpers).
//
// Layout of one item on the warp: the item's ni targets sit in
// P = ceil(ni / IB) lane slots (IB targets per lane, register-resident) and
// the warp's nsub = 32 / P lane subsets take interleaved entries of each
// staged tile, so one shared-memory read of an entry feeds IB pairs.
//
// Staging: a tile holds up to T = 32 * SPL list entries.  Every lane loads
// SPL entries (index, then the source's per-step float pair from k_split and,
// for a cell, its quadrupole), converts them to group-centre-relative FP32
// records and writes them to the warp's shared-memory tile; the tile is
// padded with zero-mass records to a multiple of 2 nsub, so every active lane
// runs the same even trip count and takes entries two at a time.  Large tiles
// keep the per-tile work (loads, conversion, two __syncwarp) small against
// the pairs; other warps cover the load latency.  No block-wide barrier.
//
// Records: a cell tile stores 48-byte records (x, y, z, m | Qxx, Qyy, Qzz,
// Qxy | Qxz, Qyz, -, -), a particle tile 16-byte records (x, y, z, m).
//
// Sums: a lane accumulates pairs in plain FP32 over a tile and adds the tile
// sum to its Kahan-compensated running sum; the lane subsets are merged with
// a compensated FP32 sum in a fixed pairwise order and converted to FP64 once.

// Resident warps per SM asked of the register allocator (more warps hide the
// latency of the staged loads).
constexpr int warp_min_blocks(int nw, int ib) { return (ib == 1 ? 24 : ib == 2 ? 20 : 12) / nw; }

template <int NW, int IB, int SPL>
__global__ void __launch_bounds__(NW * 32, warp_min_blocks(NW, IB)) k_force_warp(const otoo_dev_system sys,
                                                                                 double* __restrict__ accel,
                                                                                 double* __restrict__ pot)
{
    constexpr int T = 32 * SPL;
    __shared__ float4 s_rec[NW][3 * T];

    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    uint32_t* status = sys.counter + 1;
    const float4* __restrict__ ff = reinterpret_cast<const float4*>(sys.split);
    const bool has_quad = sys.quad != nullptr;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

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
        // records per tile are padded to a multiple of U = 2 nsub (nsub when a
        // tile holds fewer than 2 nsub records)
        const int U = T >= 2 * nsub ? 2 * nsub : nsub;
        const int TE = (T / U) * U;  // entries per tile
        const float eps2 = (float)grp.eps2;
        // the group centre rounded to FP32 (any point near the group serves)
        const float cx = __double2float_rn(grp.cx), cy = __double2float_rn(grp.cy), cz = __double2float_rn(grp.cz);

        float xi[IB], yi[IB], zi[IB];
        Acc<float> acc[IB];
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            const int i = islot + k * P;
            xi[k] = yi[k] = zi[k] = 0.f;
            if (active && i < ni) {
                const int64_t t = (int64_t)grp.first + item.i0 + i;
                const float4 h = __ldg(ff + 2 * t);
                const float4 l = __ldg(ff + 2 * t + 1);
                xi[k] = rel32(h.x, l.x, cx);
                yi[k] = rel32(h.y, l.y, cy);
                zi[k] = rel32(h.z, l.z, cz);
            }
            acc[k].zero();
        }

        // tiles: the cell entries of [j0, j1) first, then the particle entries
        const int c0 = item.j0, c1 = min(item.j1, grp.n_cell);
        const int p0 = max(item.j0, grp.n_cell), p1 = item.j1;
        const int ntc = c1 > c0 ? (c1 - c0 + TE - 1) / TE : 0;
        const int ntp = p1 > p0 ? (p1 - p0 + TE - 1) / TE : 0;
        const int nt = ntc + ntp;
        const int32_t* __restrict__ lst = sys.list + grp.list_off;
        float4* __restrict__ rec = s_rec[wid];

        // list indices of the next tile, loaded while the current one is
        // evaluated (one of the two dependent global round trips per tile)
        int nidx[SPL];
        auto load_idx = [&](int t) {
            const bool cell = t < ntc;
            const int base = cell ? c0 + t * TE : p0 + (t - ntc) * TE;
            const int cnt = cell ? min(TE, c1 - base) : min(TE, p1 - base);
#pragma unroll
            for (int e = 0; e < SPL; ++e) {
                const int k = lane + 32 * e;
                nidx[e] = k < cnt ? __ldg(lst + base + k) : 0;
            }
        };
        if (nt > 0) load_idx(0);

        for (int t = 0; t < nt; ++t) {
            const bool cell = t < ntc;
            const bool cq = cell && has_quad;
            const int base = cell ? c0 + t * TE : p0 + (t - ntc) * TE;
            const int cnt = cell ? min(TE, c1 - base) : min(TE, p1 - base);
            const int cnt_pad = (cnt + U - 1) / U * U;

            // stage: two entries per lane at a time, loads first
#pragma unroll
            for (int e0 = 0; e0 < SPL; e0 += 2) {
                float4 h[2], l[2], qa[2], qb[2];
                bool real[2], any[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int k = lane + 32 * (e0 + u);
                    real[u] = k < cnt;
                    any[u] = k < cnt_pad;
                    h[u] = l[u] = qa[u] = qb[u] = zero4;
                    if (real[u]) {
                        const int idx = nidx[e0 + u];
                        const bool good =
                            cell ? (idx >= sys.n_part && idx < sys.n_src) : (idx >= 0 && idx < sys.n_part);
                        if (good) {
                            h[u] = __ldg(ff + 2 * (int64_t)idx);
                            l[u] = __ldg(ff + 2 * (int64_t)idx + 1);
                            if (cq) {
                                const float4* qp = reinterpret_cast<const float4*>(sys.quad + (idx - sys.n_part));
                                qa[u] = __ldg(qp);
                                qb[u] = __ldg(qp + 1);
                            }
                        } else {
                            atomicOr(status, kBadIndex);
                            real[u] = false;
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (!any[u]) continue;
                    const int k = lane + 32 * (e0 + u);
                    // padding and rejected entries loaded as zeros: mass (and
                    // quadrupole) 0, so they add exactly nothing
                    const float4 a = make_float4(rel32(h[u].x, l[u].x, cx), rel32(h[u].y, l[u].y, cy),
                                                 rel32(h[u].z, l[u].z, cz), h[u].w);
                    if (cq) {
                        rec[3 * k] = a;
                        rec[3 * k + 1] = qa[u];
                        // (xz, yz, B_2 eps^2, -) for the softened quadrupole term
                        rec[3 * k + 2] = make_float4(qb[u].x, qb[u].y, qb[u].z * eps2, 0.f);
                    } else {
                        rec[k] = a;
                    }
                }
            }
            if (t + 1 < nt) load_idx(t + 1);
            __syncwarp();

            if (active) {
                float p[IB][4];
#pragma unroll
                for (int k = 0; k < IB; ++k) p[k][0] = p[k][1] = p[k][2] = p[k][3] = 0.f;
                const int niter = cnt_pad / nsub;
                if (cq) {
                    const int S = 3 * nsub;
                    const float4* __restrict__ r0 = rec + 3 * js;
                    const float4* __restrict__ r1 = r0 + S;
                    const float4* const rend = r0 + (niter & ~1) * S;
                    for (; r0 < rend; r0 += 2 * S, r1 += 2 * S) {
                        const float4 sa = r0[0], qa = r0[1], qb = r0[2];
                        const float4 sb = r1[0], qc = r1[1], qd = r1[2];
#pragma unroll
                        for (int k = 0; k < IB; ++k) {
                            pair_quad(V4<float>{sa.x, sa.y, sa.z, sa.w}, V4<float>{qa.x, qa.y, qa.z, qa.w},
                                      V4<float>{qb.x, qb.y, qb.z, qb.w}, xi[k], yi[k], zi[k], eps2, p[k]);
                            pair_quad(V4<float>{sb.x, sb.y, sb.z, sb.w}, V4<float>{qc.x, qc.y, qc.z, qc.w},
                                      V4<float>{qd.x, qd.y, qd.z, qd.w}, xi[k], yi[k], zi[k], eps2, p[k]);
                        }
                    }
                    if (niter & 1) {
                        const float4 sa = r0[0], qa = r0[1], qb = r0[2];
#pragma unroll
                        for (int k = 0; k < IB; ++k)
                            pair_quad(V4<float>{sa.x, sa.y, sa.z, sa.w}, V4<float>{qa.x, qa.y, qa.z, qa.w},
                                      V4<float>{qb.x, qb.y, qb.z, qb.w}, xi[k], yi[k], zi[k], eps2, p[k]);
                    }
                } else {
                    const float4* __restrict__ r0 = rec + js;
                    const float4* __restrict__ r1 = r0 + nsub;
                    const float4* const rend = r0 + (niter & ~1) * nsub;
                    for (; r0 < rend; r0 += 2 * nsub, r1 += 2 * nsub) {
                        const float4 sa = *r0, sb = *r1;
#pragma unroll
                        for (int k = 0; k < IB; ++k) {
                            pair_mono(V4<float>{sa.x, sa.y, sa.z, sa.w}, xi[k], yi[k], zi[k], eps2, p[k]);
                            pair_mono(V4<float>{sb.x, sb.y, sb.z, sb.w}, xi[k], yi[k], zi[k], eps2, p[k]);
                        }
                    }
                    if (niter & 1) {
                        const float4 sa = *r0;
#pragma unroll
                        for (int k = 0; k < IB; ++k)
                            pair_mono(V4<float>{sa.x, sa.y, sa.z, sa.w}, xi[k], yi[k], zi[k], eps2, p[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < IB; ++k) acc[k].add(p[k]);
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
