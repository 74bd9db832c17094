// FP32 force kernel, one work item per warp (included by force.cu, inside its
// anonymous namespace, after the pair laws and the item helpers).
//
// Layout of one item on the warp: the item's ni targets sit in
// P = ceil(ni / IB) lane slots (IB targets per lane, register-resident) and
// the warp's nsub = 32 / P lane subsets take interleaved entries of each
// staged tile, so one shared-memory read of an entry feeds IB pairs.
//
// Staging: a tile holds TE = (T / nsub) * nsub entries (T = 32 * SPL); the
// last tile of a segment is padded with zero-mass records to a multiple of
// nsub, so every active lane runs the same trip count.  Every lane converts
// SPL entries (centre-relative FP32 from the per-step float pair of k_split)
// into the warp's double buffer; the global loads of tile t+1 are issued
// before tile t is evaluated; one __syncwarp per tile, no block barrier.
//
// Records: a cell tile stores 48-byte records (x, y, z, m | Qxx, Qyy, Qzz,
// Qxy | Qxz, Qyz, -, -), a particle tile 16-byte records (x, y, z, m).
//
// Sums: a lane accumulates pairs in plain FP32 per tile and adds the tile
// sum to a Kahan-compensated running sum every FLUSH tiles; the lane subsets
// are merged with a compensated FP32 sum in subset order and converted to
// FP64 once.

#ifndef OTOO_WARP_MINB
#define OTOO_WARP_MINB 1  // minimum resident CTAs per SM requested from the register allocator
#endif
#ifndef OTOO_QUAD_UNROLL
#define OTOO_QUAD_UNROLL 2
#endif
#ifndef OTOO_MONO_UNROLL
#define OTOO_MONO_UNROLL 4
#endif
#define OTOO_PRAGMA(x) _Pragma(#x)
#define OTOO_UNROLL(n) OTOO_PRAGMA(unroll n)

template <int NW, int IB, int SPL>
__global__ void __launch_bounds__(NW * 32, OTOO_WARP_MINB) k_force_warp(const otoo_dev_system sys, double* __restrict__ accel,
                                                        double* __restrict__ pot)
{
    constexpr int T = 32 * SPL;
    constexpr int FLUSH = SPL >= 2 ? 1 : 2;
    // two buffers of T 48-byte records per warp (float4 units)
    __shared__ float4 s_rec[NW][2][3 * T];

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
        const int TE = (T / nsub) * nsub;  // entries per tile (a multiple of nsub)
        const float eps2 = (float)grp.eps2;
        // the group centre rounded to FP32 (any point near the group serves)
        const float cx = __double2float_rn(grp.cx), cy = __double2float_rn(grp.cy), cz = __double2float_rn(grp.cz);

        float xi[IB], yi[IB], zi[IB];
        Acc<float> acc[IB];
        float p[IB][4];
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            const int i = islot + k * P;
            xi[k] = yi[k] = zi[k] = 0.f;
            if (active && i < ni) {
                const int64_t t = (int64_t)grp.first + item.i0 + i;
                const float4 h = __ldg(ff + 2 * t);
                const float4 l = __ldg(ff + 2 * t + 1);
                xi[k] = (h.x - cx) + l.x;
                yi[k] = (h.y - cy) + l.y;
                zi[k] = (h.z - cz) + l.z;
            }
            acc[k].zero();
            p[k][0] = p[k][1] = p[k][2] = p[k][3] = 0.f;
        }

        // tiles: the cell entries of [j0, j1) first, then the particle entries
        const int c0 = item.j0, c1 = min(item.j1, grp.n_cell);
        const int p0 = max(item.j0, grp.n_cell), p1 = item.j1;
        const int ntc = c1 > c0 ? (c1 - c0 + TE - 1) / TE : 0;
        const int ntp = p1 > p0 ? (p1 - p0 + TE - 1) / TE : 0;
        const int nt = ntc + ntp;
        const int32_t* __restrict__ lst = sys.list + grp.list_off;

        float4 rh[SPL], rl[SPL], rqa[SPL], rqb[SPL];
        int rstate[SPL];  // 0: no record, 1: zero record (padding), 2: entry
        auto tile_base = [&](int t) { return t < ntc ? c0 + t * TE : p0 + (t - ntc) * TE; };
        auto tile_cnt = [&](int t) { return t < ntc ? min(TE, c1 - (c0 + t * TE)) : min(TE, p1 - (p0 + (t - ntc) * TE)); };
        auto fetch = [&](int t) {
            const bool cell = t < ntc;
            const int base = tile_base(t), cnt = tile_cnt(t);
            const int cnt_pad = (cnt + nsub - 1) / nsub * nsub;
#pragma unroll
            for (int e = 0; e < SPL; ++e) {
                const int k = lane + 32 * e;
                rstate[e] = k < cnt ? 2 : (k < cnt_pad ? 1 : 0);
                rh[e] = rl[e] = rqa[e] = rqb[e] = zero4;
                if (rstate[e] != 2) continue;
                const int idx = __ldg(lst + base + k);
                const bool good = cell ? (idx >= sys.n_part && idx < sys.n_src) : (idx >= 0 && idx < sys.n_part);
                if (!good) {
                    atomicOr(status, kBadIndex);
                    rstate[e] = 1;
                    continue;
                }
                rh[e] = __ldg(ff + 2 * (int64_t)idx);
                rl[e] = __ldg(ff + 2 * (int64_t)idx + 1);
                if (cell && has_quad) {
                    const float4* qp = reinterpret_cast<const float4*>(sys.quad + (idx - sys.n_part));
                    rqa[e] = __ldg(qp);
                    rqb[e] = __ldg(qp + 1);
                }
            }
        };
        auto store = [&](int t, int buf) {
            const bool cq = t < ntc && has_quad;
            float4* r = s_rec[wid][buf];
#pragma unroll
            for (int e = 0; e < SPL; ++e) {
                if (rstate[e] == 0) continue;
                const int k = lane + 32 * e;
                const float4 a = rstate[e] == 2 ? make_float4((rh[e].x - cx) + rl[e].x, (rh[e].y - cy) + rl[e].y,
                                                              (rh[e].z - cz) + rl[e].z, rh[e].w)
                                                : zero4;
                if (cq) {
                    r[3 * k] = a;
                    r[3 * k + 1] = rqa[e];
                    r[3 * k + 2] = rqb[e];
                } else {
                    r[k] = a;
                }
            }
        };

        if (nt > 0) fetch(0);
        for (int t = 0; t < nt; ++t) {
            const int buf = t & 1;
            store(t, buf);
            __syncwarp();
            const int cnt = tile_cnt(t);
            const int niter = (cnt + nsub - 1) / nsub;
            const bool cq = t < ntc && has_quad;
            if (t + 1 < nt) fetch(t + 1);
            if (active) {
                if (cq) {
                    const float4* __restrict__ r = s_rec[wid][buf] + 3 * js;
                    const int stride = 3 * nsub;
                    OTOO_UNROLL(OTOO_QUAD_UNROLL)
                    for (int n = 0; n < niter; ++n, r += stride) {
                        const float4 sv = r[0];
                        const float4 qa = r[1];
                        const float4 qb = r[2];
                        const V4<float> s4{sv.x, sv.y, sv.z, sv.w};
                        const V4<float> qa4{qa.x, qa.y, qa.z, qa.w};
                        const V2<float> qb2{qb.x, qb.y};
#pragma unroll
                        for (int k = 0; k < IB; ++k) pair_quad(s4, qa4, qb2, xi[k], yi[k], zi[k], eps2, p[k]);
                    }
                } else {
                    const float4* __restrict__ r = s_rec[wid][buf] + js;
                    OTOO_UNROLL(OTOO_MONO_UNROLL)
                    for (int n = 0; n < niter; ++n, r += nsub) {
                        const float4 sv = *r;
                        const V4<float> s4{sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                        for (int k = 0; k < IB; ++k) pair_mono(s4, xi[k], yi[k], zi[k], eps2, p[k]);
                    }
                }
                if ((t + 1) % FLUSH == 0 || t + 1 == nt) {
#pragma unroll
                    for (int k = 0; k < IB; ++k) {
                        acc[k].add(p[k]);
                        p[k][0] = p[k][1] = p[k][2] = p[k][3] = 0.f;
                    }
                }
            }
        }
        __syncwarp();

        // merge the lane subsets into the js == 0 lanes, in subset order, with
        // a compensated FP32 sum; one conversion to FP64 per output value
#pragma unroll
        for (int k = 0; k < IB; ++k) {
            double a[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float S = acc[k].s[c], C = acc[k].c[c];
                for (int j = 1; j < nsub; ++j) {
                    const float so = __shfl_sync(kFull, acc[k].s[c], islot + j * P);
                    const float co = __shfl_sync(kFull, acc[k].c[c], islot + j * P);
                    const float y = __fsub_rn(__fsub_rn(so, co), C);
                    const float t = __fadd_rn(S, y);
                    C = __fsub_rn(__fsub_rn(t, S), y);
                    S = t;
                }
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
