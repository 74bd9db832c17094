// Host half of the force step: octree, groups, interaction lists, batch
// packing and the device work plan.
//
// Paper: Section III-B (tree construction in four steps: root cube, keys,
// sort, linked cells), Section III-C (cell mass and centre of mass), Section
// III-D (vectorised group walk of Barnes 1990, the group shares one list).
// The walk runs here on the host and hands each group's list to the device.
#include <omp.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <parallel/algorithm>
#include <vector>

#include "../common.h"
#include "../plan_chunks.h"
#include "../treegeom.h"

namespace otoo {

thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

namespace {

// Allocator whose construct() default-initialises: resize() then leaves
// arithmetic elements unwritten instead of zero-filling them on one thread.
// Every array that uses it is written whole by a parallel loop right after
// its resize, which also touches its pages from the threads that use them.
template <class T>
struct NoInit : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = NoInit<U>;
    };
    NoInit() = default;
    template <class U>
    NoInit(const NoInit<U>&) noexcept
    {
    }
    template <class U, class... A>
    void construct(U* p, A&&... a)
    {
        if constexpr (sizeof...(A) == 0)
            ::new ((void*)p) U;
        else
            ::new ((void*)p) U(std::forward<A>(a)...);
    }
};
template <class T>
using filled_later = std::vector<T, NoInit<T>>;

// (Hilbert key, caller index), ordered by key then index: the sort of
// Section III-B.
struct KeyIndex {
    uint64_t key;
    int64_t index;
    bool operator<(const KeyIndex& o) const { return key < o.key || (key == o.key && index < o.index); }
};

struct Cell {
    int64_t begin, end;     // tree-order particle range
    int64_t child0;         // first child cell (children are consecutive)
    int32_t level, nchild;
};

}  // namespace
}  // namespace otoo

using namespace otoo;

struct otoo_tree {
    int64_t n = 0;
    int leaf_size = 8;
    int depth = 0;
    double lo[3] = {0, 0, 0}, S = 1, h = 1;
    otoo::filled_later<double> pos;        // [n][3] tree order
    otoo::filled_later<float> mass;        // [n]
    otoo::filled_later<int64_t> perm;      // tree -> caller index
    otoo::filled_later<uint64_t> key;      // [n]
    otoo::filled_later<int32_t> gq;        // [n][3] quantised coordinates
    std::vector<otoo::Cell> cells;
    // flat per-cell arrays (exported, and used by the walk)
    otoo::filled_later<int64_t> c_begin, c_end, c_child0, c_org;
    otoo::filled_later<int32_t> c_level, c_nchild;
    otoo::filled_later<double> c_com, c_mass, c_quad;     // [3], [1], [6]
    otoo::filled_later<double> c_b2, c_bmax;               // spread about the centre of mass (Eq. B2)
    otoo::filled_later<double> c_lo, c_side, c_gc;         // cube lower corner [3], side, centre [3]
};

struct otoo_lists {
    int64_t n_part = 0, n_src = 0;
    int32_t n_sys = 1, use_quad = 0;
    otoo::filled_later<otoo_src> src;      // written whole by fill_sources / the batch copy
    otoo::filled_later<otoo_quad> quad;
    std::vector<otoo_group> groups;
    otoo::filled_later<int32_t> list;      // written whole by the per-group copies
    std::vector<int64_t> perm;
    std::vector<int64_t> sys_part_off;
    int64_t interactions = 0, cell_interactions = 0;
    double eps = 0;
};

struct otoo_plan {
    std::vector<otoo_item> items;
    std::vector<otoo_split> splits;
    int64_t partial_doubles = 0;
    int32_t n_crit_max = 0;
};

namespace {

template <class F>
int guarded(F&& f)
{
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return set_error(OTOO_ENOMEM, "host allocation failed");
    } catch (...) {
        return set_error(OTOO_EINVAL, "unexpected host error");
    }
}

// Cell moments by direct summation over the cell's particle range (the
// "direct summation for each cell" variant of Section III-C; it parallelises
// over cells): mass, centre of mass, traceless quadrupole about it, and the
// spread the absolute MAC needs: B_2 = sum m |com - x|^2 (Eq. B2) and
// b_max = max |com - x|.
void cell_moments(otoo_tree* t, int64_t c)
{
    const int64_t b = t->c_begin[c], e = t->c_end[c];
    double m = 0, sx = 0, sy = 0, sz = 0;
    for (int64_t i = b; i < e; ++i) {
        const double mi = t->mass[i];
        m += mi;
        sx += mi * t->pos[3 * i];
        sy += mi * t->pos[3 * i + 1];
        sz += mi * t->pos[3 * i + 2];
    }
    const double cx = sx / m, cy = sy / m, cz = sz / m;
    double q[6] = {0, 0, 0, 0, 0, 0};
    double b2 = 0, dmax2 = 0;
    for (int64_t i = b; i < e; ++i) {
        const double mi = t->mass[i];
        const double dx = t->pos[3 * i] - cx, dy = t->pos[3 * i + 1] - cy, dz = t->pos[3 * i + 2] - cz;
        const double d2 = dx * dx + dy * dy + dz * dz;
        b2 += mi * d2;
        dmax2 = std::max(dmax2, d2);
        q[0] += mi * (3 * dx * dx - d2);
        q[1] += mi * (3 * dy * dy - d2);
        q[2] += mi * (3 * dz * dz - d2);
        q[3] += mi * 3 * dx * dy;
        q[4] += mi * 3 * dx * dz;
        q[5] += mi * 3 * dy * dz;
    }
    t->c_mass[c] = m;
    t->c_com[3 * c] = cx;
    t->c_com[3 * c + 1] = cy;
    t->c_com[3 * c + 2] = cz;
    for (int k = 0; k < 6; ++k) t->c_quad[6 * c + k] = q[k];
    t->c_b2[c] = b2;
    t->c_bmax[c] = std::sqrt(dmax2);
    // cube geometry on the grid: side h 2^(21-L), lower corner lo + org h
    const double side = cube_side(t->h, t->c_level[c]);
    t->c_side[c] = side;
    for (int a = 0; a < 3; ++a) {
        t->c_lo[3 * c + a] = cube_lo(t->lo[a], t->c_org[3 * c + a], t->h);
        t->c_gc[3 * c + a] = cube_centre(t->c_lo[3 * c + a], side);
    }
}

// Build the cell hierarchy from the sorted keys (Section III-B, last step):
// a cell holding more than leaf_size particles (and above the last grid
// level) is sliced into the runs of equal 3-bit key digit of the next level.
void build_cells(otoo_tree* t)
{
    std::vector<Cell>& cells = t->cells;
    cells.clear();
    cells.push_back(Cell{0, t->n, -1, 0, 0});
    std::vector<int64_t> stack{0};
    int depth = 0;
    while (!stack.empty()) {
        const int64_t c = stack.back();
        stack.pop_back();
        const Cell cc = cells[c];
        depth = std::max(depth, cc.level);
        if (cc.end - cc.begin <= t->leaf_size || cc.level == kLevels) continue;
        const int shift = 3 * (kLevels - 1 - cc.level);
        const int64_t child0 = (int64_t)cells.size();
        int nchild = 0;
        int64_t b = cc.begin;
        while (b < cc.end) {
            const uint64_t d = (t->key[b] >> shift) & 7u;
            // first particle of the next digit run (keys sorted within the cell)
            const uint64_t* kb = t->key.data() + b;
            const uint64_t* ke = t->key.data() + cc.end;
            const uint64_t* it = std::partition_point(kb, ke, [&](uint64_t k) { return ((k >> shift) & 7u) <= d; });
            const int64_t e = b + (it - kb);
            cells.push_back(Cell{b, e, -1, cc.level + 1, 0});
            ++nchild;
            b = e;
        }
        cells[c].child0 = child0;
        cells[c].nchild = nchild;
        for (int k = nchild - 1; k >= 0; --k) stack.push_back(child0 + k);
    }
    t->depth = depth;
    const int64_t nc = (int64_t)cells.size();
    t->c_begin.resize(nc);
    t->c_end.resize(nc);
    t->c_child0.resize(nc);
    t->c_org.resize(3 * nc);
    t->c_level.resize(nc);
    t->c_nchild.resize(nc);
    t->c_com.resize(3 * nc);
    t->c_mass.resize(nc);
    t->c_quad.resize(6 * nc);
    t->c_b2.resize(nc);
    t->c_bmax.resize(nc);
    t->c_lo.resize(3 * nc);
    t->c_side.resize(nc);
    t->c_gc.resize(3 * nc);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t c = 0; c < nc; ++c) {
        const Cell& cc = cells[c];
        t->c_begin[c] = cc.begin;
        t->c_end[c] = cc.end;
        t->c_child0[c] = cc.child0;
        t->c_level[c] = cc.level;
        t->c_nchild[c] = cc.nchild;
        const int sh = kLevels - cc.level;
        for (int a = 0; a < 3; ++a) {
            const int64_t g = t->gq[3 * cc.begin + a];
            t->c_org[3 * c + a] = sh >= kLevels ? 0 : (g >> sh) << sh;
        }
        cell_moments(t, c);
    }
}

}  // namespace

extern "C" {

const char* otoo_last_error(void) { return g_last_error.c_str(); }

int otoo_build_tree(const double* pos, const float* mass, int64_t n, const otoo_params* params,
                    otoo_tree** out)
{
    Range range_("otoo_build_tree");
    OTOO_REQUIRE(out != nullptr, OTOO_EINVAL, "otoo_build_tree: out is NULL");
    *out = nullptr;
    OTOO_REQUIRE(pos && mass && params, OTOO_EINVAL, "otoo_build_tree: NULL input");
    OTOO_REQUIRE(n >= 1 && n <= ((int64_t)1 << 30), OTOO_EINVAL, "otoo_build_tree: n = %lld out of range",
                 (long long)n);
    OTOO_REQUIRE(params->leaf_size >= 1, OTOO_EINVAL, "otoo_build_tree: leaf_size < 1");
    return guarded([&]() -> int {
        int bad = 0;
#pragma omp parallel for reduction(| : bad)
        for (int64_t i = 0; i < n; ++i) {
            if (!std::isfinite(pos[3 * i]) || !std::isfinite(pos[3 * i + 1]) || !std::isfinite(pos[3 * i + 2]) ||
                !(mass[i] > 0.0f) || !std::isfinite(mass[i]))
                bad |= 1;
        }
        OTOO_REQUIRE(!bad, OTOO_EINVAL, "otoo_build_tree: non-finite position or mass <= 0");
        otoo_tree* t = new otoo_tree();
        t->n = n;
        t->leaf_size = params->leaf_size;
        // step 1: root cube
        double mn[3] = {pos[0], pos[1], pos[2]}, mx[3] = {pos[0], pos[1], pos[2]};
#pragma omp parallel
        {
            double lmn[3] = {pos[0], pos[1], pos[2]}, lmx[3] = {pos[0], pos[1], pos[2]};
#pragma omp for nowait
            for (int64_t i = 0; i < n; ++i)
                for (int a = 0; a < 3; ++a) {
                    lmn[a] = std::min(lmn[a], pos[3 * i + a]);
                    lmx[a] = std::max(lmx[a], pos[3 * i + a]);
                }
#pragma omp critical
            for (int a = 0; a < 3; ++a) {
                mn[a] = std::min(mn[a], lmn[a]);
                mx[a] = std::max(mx[a], lmx[a]);
            }
        }
        root_cube(mn, mx, t->lo, &t->S, &t->h);
        const double scale = kGrid / t->S;
        // step 2: quantise and key
        filled_later<KeyIndex> kv(n);
        filled_later<int32_t> gq0(3 * n);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            uint32_t g[3];
            for (int a = 0; a < 3; ++a) {
                g[a] = quantize(pos[3 * i + a], t->lo[a], scale);
                gq0[3 * i + a] = (int32_t)g[a];
            }
            kv[i] = KeyIndex{hilbert_key(g[0], g[1], g[2]), i};
        }
        // step 3: sort (key, index) -- libstdc++ parallel mode, as in the paper
        __gnu_parallel::sort(kv.begin(), kv.end());
        t->pos.resize(3 * n);
        t->mass.resize(n);
        t->perm.resize(n);
        t->key.resize(n);
        t->gq.resize(3 * n);
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < n; ++k) {
            const int64_t i = kv[k].index;
            t->perm[k] = i;
            t->key[k] = kv[k].key;
            t->mass[k] = mass[i];
            for (int a = 0; a < 3; ++a) {
                t->pos[3 * k + a] = pos[3 * i + a];
                t->gq[3 * k + a] = gq0[3 * i + a];
            }
        }
        // step 4: cells and their properties
        build_cells(t);
        *out = t;
        return OTOO_OK;
    });
}

int otoo_tree_export(const otoo_tree* t, otoo_tree_view* v)
{
    OTOO_REQUIRE(t && v, OTOO_EINVAL, "otoo_tree_export: NULL argument");
    v->n_part = t->n;
    v->n_cell = (int64_t)t->cells.size();
    v->depth = t->depth;
    v->leaf_size = t->leaf_size;
    for (int a = 0; a < 3; ++a) v->root_lo[a] = t->lo[a];
    v->root_side = t->S;
    v->pos = t->pos.data();
    v->mass = t->mass.data();
    v->perm = t->perm.data();
    v->cell_begin = t->c_begin.data();
    v->cell_end = t->c_end.data();
    v->cell_level = t->c_level.data();
    v->cell_nchild = t->c_nchild.data();
    v->cell_child0 = t->c_child0.data();
    v->cell_org = t->c_org.data();
    v->cell_com = t->c_com.data();
    v->cell_mass = t->c_mass.data();
    v->cell_quad = t->c_quad.data();
    v->cell_b2 = t->c_b2.data();
    v->cell_bmax = t->c_bmax.data();
    return OTOO_OK;
}

void otoo_tree_free(otoo_tree* t) { delete t; }

}  // extern "C"

namespace {

struct GroupRange {
    int64_t begin, end;
};

// Groups: the maximal cells with at most n_crit particles, in tree order.  A
// leaf on the last grid level with more than n_crit particles (coincident
// points) is cut into consecutive chunks of n_crit.
void find_groups(const otoo_tree* t, int n_crit, std::vector<GroupRange>& out)
{
    std::vector<int64_t> stack{0};
    while (!stack.empty()) {
        const int64_t c = stack.back();
        stack.pop_back();
        const int64_t b = t->c_begin[c], e = t->c_end[c];
        if (e - b <= n_crit) {
            out.push_back({b, e});
        } else if (t->c_nchild[c] == 0) {
            for (int64_t s = b; s < e; s += n_crit) out.push_back({s, std::min(e, s + n_crit)});
        } else {
            for (int k = t->c_nchild[c] - 1; k >= 0; --k) stack.push_back(t->c_child0[c] + k);
        }
    }
}

// s = |com - cube centre| of every cell (Section II-B), once per walk.
void cell_offsets(const otoo_tree* t, std::vector<double>& s)
{
    const int64_t nc = (int64_t)t->cells.size();
    s.resize(nc);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        double s2 = 0;
        for (int a = 0; a < 3; ++a) {
            const double e = t->c_com[3 * c + a] - t->c_gc[3 * c + a];
            s2 += e * e;
        }
        s[c] = std::sqrt(s2);
    }
}

// Group MAC: accept cell c for the box [blo, bhi] when the cube misses the
// box and d_min > l / theta + s (notation of Section II-B); thr = l / theta +
// s comes from the caller (side / theta, then + s, in FP64).
inline bool mac_accept(const otoo_tree* t, int64_t c, const double blo[3], const double bhi[3], double thr)
{
    const double side = t->c_side[c];
    const double* clo = &t->c_lo[3 * c];
    if (clo[0] <= bhi[0] && blo[0] <= clo[0] + side && clo[1] <= bhi[1] && blo[1] <= clo[1] + side &&
        clo[2] <= bhi[2] && blo[2] <= clo[2] + side)
        return false;
    const double* com = &t->c_com[3 * c];
    double d2 = 0;
    for (int a = 0; a < 3; ++a) {
        double d = 0;
        if (blo[a] - com[a] > d) d = blo[a] - com[a];
        if (com[a] - bhi[a] > d) d = com[a] - bhi[a];
        d2 += d * d;
    }
    return std::sqrt(d2) > thr;
}

// Absolute MAC for the box [blo, bhi]: d_min (centre of mass to the box) > r_b.
inline bool sw_accept(const otoo_tree* t, int64_t c, const double blo[3], const double bhi[3], double rb)
{
    const double* com = &t->c_com[3 * c];
    double d2 = 0;
    for (int a = 0; a < 3; ++a) {
        double d = 0;
        if (blo[a] - com[a] > d) d = blo[a] - com[a];
        if (com[a] - bhi[a] > d) d = com[a] - bhi[a];
        d2 += d * d;
    }
    return std::sqrt(d2) > rb;
}

// SPH bounding radius of every cell (Eq. SPH_RAD): the largest |com - x_j| +
// h_j over the cell's particles (h in caller order).
void sph_radii(const otoo_tree* t, const float* h, std::vector<double>& rb)
{
    const int64_t nc = (int64_t)t->cells.size();
    rb.resize(nc);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t c = 0; c < nc; ++c) {
        const double* com = &t->c_com[3 * c];
        double r = 0;
        for (int64_t j = t->c_begin[c]; j < t->c_end[c]; ++j) {
            const double dx = com[0] - t->pos[3 * j], dy = com[1] - t->pos[3 * j + 1], dz = com[2] - t->pos[3 * j + 2];
            const double v = std::sqrt(dx * dx + dy * dy + dz * dz) + (double)h[t->perm[j]];
            if (v > r) r = v;
        }
        rb[c] = r;
    }
}

bool valid_h(const float* h, int64_t n)
{
    if (!h) return false;
    for (int64_t i = 0; i < n; ++i)
        if (!(h[i] > 0.0f) || !std::isfinite(h[i])) return false;
    return true;
}

// Sources of the force step: particles in tree order, then cells (centre of
// mass, mass) and their quadrupoles (zeros for monopole cells).
void fill_sources(const otoo_tree* t, int use_quad, otoo_src* src, otoo_quad* quad)
{
    const int64_t n = t->n, nc = (int64_t)t->cells.size();
    if (src) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            otoo_src& s = src[i];
            s.x = t->pos[3 * i];
            s.y = t->pos[3 * i + 1];
            s.z = t->pos[3 * i + 2];
            s.m = t->mass[i];
            s.pad = 0;
        }
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < nc; ++c) {
            otoo_src& s = src[n + c];
            s.x = t->c_com[3 * c];
            s.y = t->c_com[3 * c + 1];
            s.z = t->c_com[3 * c + 2];
            s.m = (float)t->c_mass[c];
            s.pad = 0;
        }
    }
    if (quad) {
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < nc; ++c) {
            otoo_quad& q = quad[c];
            const double* qq = &t->c_quad[6 * c];
            const bool u = use_quad != 0;
            q.xx = u ? (float)qq[0] : 0.f;
            q.yy = u ? (float)qq[1] : 0.f;
            q.zz = u ? (float)qq[2] : 0.f;
            q.xy = u ? (float)qq[3] : 0.f;
            q.xz = u ? (float)qq[4] : 0.f;
            q.yz = u ? (float)qq[5] : 0.f;
            q.b2 = u ? (float)t->c_b2[c] : 0.f;
            q.pad = 0.f;
        }
    }
}

}  // namespace

extern "C" {

int otoo_make_groups_and_lists(const otoo_tree* t, const otoo_params* p, otoo_lists** out)
{
    Range range_("otoo_make_groups_and_lists");
    OTOO_REQUIRE(out != nullptr, OTOO_EINVAL, "otoo_make_groups_and_lists: out is NULL");
    *out = nullptr;
    OTOO_REQUIRE(t && p, OTOO_EINVAL, "otoo_make_groups_and_lists: NULL argument");
    OTOO_REQUIRE(p->eps > 0.0 && std::isfinite(p->eps), OTOO_EINVAL, "eps must be > 0");
    OTOO_REQUIRE(p->n_crit >= 1 && p->n_crit <= kMaxGroup, OTOO_EINVAL, "n_crit out of [1, %d]", kMaxGroup);
    OTOO_REQUIRE(p->theta >= 0.0 && std::isfinite(p->theta), OTOO_EINVAL, "theta must be finite and >= 0");
    OTOO_REQUIRE(p->mac == OTOO_MAC_THETA || p->mac == OTOO_MAC_SW || p->mac == OTOO_MAC_SPH, OTOO_EINVAL,
                 "unknown mac %d", p->mac);
    OTOO_REQUIRE(p->mac != OTOO_MAC_SPH || valid_h(p->h_sph, t->n), OTOO_EINVAL,
                 "OTOO_MAC_SPH needs h_sph > 0 and finite for every particle");
    OTOO_REQUIRE(p->mac != OTOO_MAC_SW || (p->delta >= 0.0 && std::isfinite(p->delta) && std::isfinite(p->m_limit)),
                 OTOO_EINVAL, "delta must be finite and >= 0, m_limit finite");
    OTOO_REQUIRE(t->n <= INT32_MAX / 2, OTOO_EINVAL, "too many particles for 32-bit list indices");
    return guarded([&]() -> int {
        std::vector<GroupRange> gr;
        find_groups(t, p->n_crit, gr);
        const int64_t G = (int64_t)gr.size();
        OTOO_REQUIRE(G <= INT32_MAX, OTOO_EINVAL, "too many groups");
        if (p->theta_per_group) {
            for (int64_t g = 0; g < G; ++g)
                OTOO_REQUIRE(std::isfinite(p->theta_per_group[g]), OTOO_EINVAL, "theta_per_group[%lld] not finite",
                             (long long)g);
        }
        otoo_lists* L = new otoo_lists();
        const int64_t n = t->n, nc = (int64_t)t->cells.size();
        L->n_part = n;
        L->n_src = n + nc;
        L->use_quad = p->use_quad ? 1 : 0;
        L->eps = p->eps;
        L->groups.resize(G);
        const bool sw = p->mac == OTOO_MAC_SW, sph = p->mac == OTOO_MAC_SPH;
        std::vector<double> rb;
        if (sw) {
            rb.resize(nc);
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < nc; ++c)
                rb[c] = sw_radius(t->c_b2[c], t->c_bmax[c], t->c_mass[c], p->delta, p->m_limit, t->S);
        } else if (sph) {
            sph_radii(t, p->h_sph, rb);
        }
        // opening angle: s of every cell once, and with one angle for all
        // groups the threshold l / theta + s too
        std::vector<double> cs, thr;
        if (!sw && !sph) {
            cell_offsets(t, cs);
            if (!p->theta_per_group && p->theta > 0.0) {
                thr.resize(nc);
#pragma omp parallel for schedule(static)
                for (int64_t c = 0; c < nc; ++c) thr[c] = t->c_side[c] / p->theta + cs[c];
            }
        }
        // the walk: one shared list per group (Barnes 1990, Section III-D),
        // entries buffered per thread, then placed in group order
        const int nthr = omp_get_max_threads();
        std::vector<std::vector<int32_t>> tbuf(nthr);
        std::vector<int64_t> goff(G), gthr(G);
#pragma omp parallel
        {
            const int tid = omp_get_thread_num();
            std::vector<int32_t>& buf = tbuf[tid];
            std::vector<int64_t> stack;
            std::vector<int32_t> parts;
#pragma omp for schedule(dynamic, 16)
            for (int64_t g = 0; g < G; ++g) {
                const int64_t b = gr[g].begin, e = gr[g].end;
                double blo[3], bhi[3];
                for (int a = 0; a < 3; ++a) blo[a] = bhi[a] = t->pos[3 * b + a];
                for (int64_t i = b + 1; i < e; ++i)
                    for (int a = 0; a < 3; ++a) {
                        blo[a] = std::min(blo[a], t->pos[3 * i + a]);
                        bhi[a] = std::max(bhi[a], t->pos[3 * i + a]);
                    }
                const double theta = (sw || sph) ? 0.0 : p->theta_per_group ? (double)p->theta_per_group[g] : p->theta;
                const int64_t start = (int64_t)buf.size();
                parts.clear();
                stack.clear();
                if (theta >= 0.0) stack.push_back(0);  // a negative angle skips the group
                int64_t ncell = 0;
                while (!stack.empty()) {
                    const int64_t c = stack.back();
                    stack.pop_back();
                    if (sph) {
                        // no neighbour of the group in c: skip it (Eq. SPH_RAD)
                        if (sw_accept(t, c, blo, bhi, rb[c])) continue;
                        if (t->c_nchild[c] == 0) {
                            for (int64_t i = t->c_begin[c]; i < t->c_end[c]; ++i) parts.push_back((int32_t)i);
                        } else {
                            const int64_t c0 = t->c_child0[c];
                            for (int k = t->c_nchild[c] - 1; k >= 0; --k) stack.push_back(c0 + k);
                        }
                    } else if (sw ? sw_accept(t, c, blo, bhi, rb[c])
                                  : theta > 0.0 &&
                                        mac_accept(t, c, blo, bhi,
                                                   thr.empty() ? t->c_side[c] / theta + cs[c] : thr[c])) {
                        buf.push_back((int32_t)(n + c));
                        ++ncell;
                    } else if (t->c_nchild[c] == 0) {
                        for (int64_t i = t->c_begin[c]; i < t->c_end[c]; ++i) parts.push_back((int32_t)i);
                    } else {
                        const int64_t c0 = t->c_child0[c];
                        for (int k = t->c_nchild[c] - 1; k >= 0; --k) stack.push_back(c0 + k);
                    }
                }
                // particle entries in increasing tree order after the cells (the
                // pre-order walk meets the leaves in tree order already)
                if (!std::is_sorted(parts.begin(), parts.end())) std::sort(parts.begin(), parts.end());
                buf.insert(buf.end(), parts.begin(), parts.end());
                otoo_group& og = L->groups[g];
                og.first = (int32_t)b;
                og.count = (int32_t)(e - b);
                og.n_cell = (int32_t)ncell;
                og.n_part = (int32_t)parts.size();
                og.eps2 = p->eps * p->eps;
                og.cx = (blo[0] + bhi[0]) * 0.5;
                og.cy = (blo[1] + bhi[1]) * 0.5;
                og.cz = (blo[2] + bhi[2]) * 0.5;
                og.theta = (float)theta;
                og.sys = 0;
                goff[g] = start;
                gthr[g] = tid;
            }
        }
        int64_t total = 0, inter = 0, cinter = 0;
        std::vector<int64_t> dst(G);
        for (int64_t g = 0; g < G; ++g) {
            otoo_group& og = L->groups[g];
            dst[g] = total;
            og.list_off = total;
            total += og.n_cell + og.n_part;
            inter += (int64_t)og.count * (og.n_cell + og.n_part);
            cinter += (int64_t)og.count * og.n_cell;
        }
        L->list.resize(total);
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t g = 0; g < G; ++g) {
            const otoo_group& og = L->groups[g];
            const int32_t* s = tbuf[gthr[g]].data() + goff[g];
            std::memcpy(L->list.data() + dst[g], s, sizeof(int32_t) * (size_t)(og.n_cell + og.n_part));
        }
        tbuf.clear();
        L->interactions = inter;
        L->cell_interactions = cinter;
        L->src.resize(n + nc);
        L->quad.resize(nc);
        fill_sources(t, L->use_quad, L->src.data(), L->quad.data());
        L->perm.assign(t->perm.begin(), t->perm.end());
        L->sys_part_off = {0, n};
        *out = L;
        return OTOO_OK;
    });
}

int otoo_lists_export(const otoo_lists* L, otoo_lists_view* v)
{
    OTOO_REQUIRE(L && v, OTOO_EINVAL, "otoo_lists_export: NULL argument");
    v->n_part = L->n_part;
    v->n_src = L->n_src;
    v->n_groups = (int64_t)L->groups.size();
    v->n_list = (int64_t)L->list.size();
    v->n_sys = L->n_sys;
    v->use_quad = L->use_quad;
    v->src = L->src.data();
    v->quad = L->quad.data();
    v->groups = L->groups.data();
    v->list = L->list.data();
    v->perm = L->perm.data();
    v->sys_part_off = L->sys_part_off.data();
    v->interactions = L->interactions;
    v->cell_interactions = L->cell_interactions;
    return OTOO_OK;
}

void otoo_lists_free(otoo_lists* L) { delete L; }

int otoo_find_groups(const otoo_tree* t, int32_t n_crit, int32_t* first, int32_t* count, int64_t capacity,
                     int64_t* n_groups)
{
    OTOO_REQUIRE(t && n_groups, OTOO_EINVAL, "otoo_find_groups: NULL argument");
    OTOO_REQUIRE(n_crit >= 1 && n_crit <= kMaxGroup, OTOO_EINVAL, "n_crit out of [1, %d]", kMaxGroup);
    OTOO_REQUIRE(capacity >= 0, OTOO_EINVAL, "otoo_find_groups: negative capacity");
    return guarded([&]() -> int {
        std::vector<GroupRange> gr;
        find_groups(t, n_crit, gr);
        const int64_t G = (int64_t)gr.size();
        *n_groups = G;
        if (!first && !count && capacity == 0) return OTOO_OK;
        OTOO_REQUIRE(first && count, OTOO_EINVAL, "otoo_find_groups: first/count NULL with capacity %lld",
                     (long long)capacity);
        OTOO_REQUIRE(G <= capacity, OTOO_EINVAL, "otoo_find_groups: %lld groups, capacity %lld", (long long)G,
                     (long long)capacity);
        for (int64_t g = 0; g < G; ++g) {
            first[g] = (int32_t)gr[g].begin;
            count[g] = (int32_t)(gr[g].end - gr[g].begin);
        }
        return OTOO_OK;
    });
}

// Walk records: the FP32 filter data (centre of mass as a float pair, its
// offset from the cube's lower corner, side, and the centre-of-mass offset s
// computed with the host test's FP64 operations) and the FP64 geometry the
// exact test reads.
int otoo_tree_device_arrays(const otoo_tree* t, int32_t use_quad, const otoo_params* p, otoo_src* src,
                            otoo_quad* quad, otoo_wcell* cell, otoo_wcell64* cell64)
{
    Range range_("otoo_tree_device_arrays");
    OTOO_REQUIRE(t, OTOO_EINVAL, "otoo_tree_device_arrays: NULL tree");
    const bool sw = p && p->mac == OTOO_MAC_SW, sph = p && p->mac == OTOO_MAC_SPH;
    OTOO_REQUIRE(!p || p->mac == OTOO_MAC_THETA || sw || sph, OTOO_EINVAL, "unknown mac %d", p ? p->mac : 0);
    OTOO_REQUIRE(!sph || valid_h(p->h_sph, t->n), OTOO_EINVAL, "OTOO_MAC_SPH needs h_sph > 0 for every particle");
    OTOO_REQUIRE(!sw || (p->delta >= 0.0 && std::isfinite(p->delta) && std::isfinite(p->m_limit)), OTOO_EINVAL,
                 "delta must be finite and >= 0, m_limit finite");
    OTOO_REQUIRE(t->n <= INT32_MAX / 2 && (int64_t)t->cells.size() <= INT32_MAX / 2, OTOO_EINVAL,
                 "otoo_tree_device_arrays: tree too large for 32-bit indices");
    return guarded([&]() -> int {
        fill_sources(t, use_quad, src, quad);
        const int64_t nc = (int64_t)t->cells.size();
        std::vector<double> rb(nc, 0.0);
        if (sw) {
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < nc; ++c)
                rb[c] = sw_radius(t->c_b2[c], t->c_bmax[c], t->c_mass[c], p->delta, p->m_limit, t->S);
        } else if (sph) {
            sph_radii(t, p->h_sph, rb);
        }
        if (cell) {
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < nc; ++c) {
                otoo_wcell& w = cell[c];
                wcell_geometry(&t->c_com[3 * c], &t->c_lo[3 * c], &t->c_gc[3 * c], t->c_side[c], &w);
                w.nchild = t->c_nchild[c];
                w.child0 = w.nchild > 0 ? (int32_t)t->c_child0[c] : 0;
                w.begin = (int32_t)t->c_begin[c];
                w.end = (int32_t)t->c_end[c];
                w.rb = (float)rb[c];
            }
        }
        if (cell64) {
#pragma omp parallel for schedule(static)
            for (int64_t c = 0; c < nc; ++c) {
                otoo_wcell64& w = cell64[c];
                for (int a = 0; a < 3; ++a) {
                    w.lo[a] = t->c_lo[3 * c + a];
                    w.com[a] = t->c_com[3 * c + a];
                    w.gc[a] = t->c_gc[3 * c + a];
                }
                w.side = t->c_side[c];
                w.rb = rb[c];
                w.pad = 0.0;
            }
        }
        return OTOO_OK;
    });
}

int otoo_pack_batch(const otoo_lists* const* per, int32_t n_sys, otoo_lists** out)
{
    Range range_("otoo_pack_batch");
    OTOO_REQUIRE(out != nullptr, OTOO_EINVAL, "otoo_pack_batch: out is NULL");
    *out = nullptr;
    OTOO_REQUIRE(per && n_sys >= 1, OTOO_EINVAL, "otoo_pack_batch: need at least one system");
    for (int k = 0; k < n_sys; ++k) OTOO_REQUIRE(per[k], OTOO_EINVAL, "otoo_pack_batch: system %d is NULL", k);
    return guarded([&]() -> int {
        otoo_lists* B = new otoo_lists();
        std::vector<int64_t> pb(n_sys + 1, 0), cb(n_sys + 1, 0), lb(n_sys + 1, 0), gb(n_sys + 1, 0);
        int any_quad = 0;
        for (int k = 0; k < n_sys; ++k) {
            const otoo_lists* s = per[k];
            pb[k + 1] = pb[k] + s->n_part;
            cb[k + 1] = cb[k] + (s->n_src - s->n_part);
            lb[k + 1] = lb[k] + (int64_t)s->list.size();
            gb[k + 1] = gb[k] + (int64_t)s->groups.size();
            any_quad |= s->use_quad;
        }
        const int64_t P = pb[n_sys], C = cb[n_sys];
        OTOO_REQUIRE(P + C <= INT32_MAX && gb[n_sys] <= INT32_MAX, OTOO_EINVAL, "batch too large for 32-bit indices");
        B->n_part = P;
        B->n_src = P + C;
        B->n_sys = n_sys;
        B->use_quad = any_quad;
        B->src.resize(P + C);
        B->quad.resize(C);
        B->groups.resize(gb[n_sys]);
        B->list.resize(lb[n_sys]);
        B->perm.resize(P);
        B->sys_part_off.assign(pb.begin(), pb.end());
#pragma omp parallel for schedule(dynamic, 1)
        for (int k = 0; k < n_sys; ++k) {
            const otoo_lists* s = per[k];
            const int64_t np = s->n_part, ncs = s->n_src - s->n_part;
            std::copy(s->src.begin(), s->src.begin() + np, B->src.begin() + pb[k]);
            std::copy(s->src.begin() + np, s->src.end(), B->src.begin() + P + cb[k]);
            if (s->use_quad)
                std::copy(s->quad.begin(), s->quad.end(), B->quad.begin() + cb[k]);
            else
                std::fill(B->quad.begin() + cb[k], B->quad.begin() + cb[k] + ncs, otoo_quad{});
            for (int64_t i = 0; i < np; ++i) B->perm[pb[k] + i] = pb[k] + s->perm[i];
            for (size_t g = 0; g < s->groups.size(); ++g) {
                otoo_group og = s->groups[g];
                og.first += (int32_t)pb[k];
                og.list_off += lb[k];
                og.sys = k;
                B->groups[gb[k] + g] = og;
            }
            for (size_t j = 0; j < s->list.size(); ++j) {
                const int64_t idx = s->list[j];
                B->list[lb[k] + j] = (int32_t)(idx < np ? pb[k] + idx : P + cb[k] + (idx - np));
            }
        }
        for (int k = 0; k < n_sys; ++k) {
            B->interactions += per[k]->interactions;
            B->cell_interactions += per[k]->cell_interactions;
        }
        *out = B;
        return OTOO_OK;
    });
}

int otoo_default_tune(int32_t n_crit, otoo_tune* tune)
{
    OTOO_REQUIRE(tune, OTOO_EINVAL, "otoo_default_tune: NULL");
    OTOO_REQUIRE(n_crit >= 1 && n_crit <= kMaxGroup, OTOO_EINVAL, "n_crit out of range");
    tune->block = 128;
    tune->iblock = 2;
    tune->tile = 128;
    tune->split = 4096;
    tune->ctas_per_sm = 0;
    tune->packed = 0;
    return OTOO_OK;
}

// Work items (longest processing time first): each group cut into particle
// chunks that fill a warp's lanes (plan_chunks.h) times list chunks of at most
// `split` entries, balanced in length.
int otoo_make_plan(const otoo_lists* L, const otoo_tune* tune, otoo_plan** out)
{
    Range range_("otoo_make_plan");
    OTOO_REQUIRE(out != nullptr, OTOO_EINVAL, "otoo_make_plan: out is NULL");
    *out = nullptr;
    OTOO_REQUIRE(L && tune, OTOO_EINVAL, "otoo_make_plan: NULL argument");
    OTOO_REQUIRE(tune->split >= 1, OTOO_EINVAL, "split must be >= 1");
    return guarded([&]() -> int {
        otoo_plan* P = new otoo_plan();
        int32_t ncm = 1;
        for (const otoo_group& g : L->groups) ncm = std::max(ncm, g.count);
        if (ncm > kMaxGroup) {
            delete P;
            return set_error(OTOO_EINVAL, "otoo_make_plan: a group holds more than %d particles", kMaxGroup);
        }
        P->n_crit_max = ncm;
        const int32_t ib = std::max(1, tune->iblock);
        // particle chunks of each group: the cut of plan_chunks.h (warp-filling
        // item sizes), the same on the device plan
        ChunkTable tab;
        chunk_table_build(ib, tab);
        int64_t slot = 0;
        for (size_t g = 0; g < L->groups.size(); ++g) {
            const otoo_group& og = L->groups[g];
            const int64_t len = (int64_t)og.n_cell + og.n_part;
            if (len == 0) continue;  // skipped group
            const int64_t nch = (len + tune->split - 1) / tune->split;
            if (nch > 1) P->splits.push_back({(int32_t)g, (int32_t)slot, (int32_t)nch, 0});
            int32_t i0 = 0;
            for (int32_t rest = og.count; rest > 0;) {
                const int32_t ni = tab.last[rest];
                for (int64_t k = 0; k < nch; ++k) {
                    const int64_t j0 = len * k / nch, j1 = len * (k + 1) / nch;
                    P->items.push_back({(int32_t)g, i0, ni, (int32_t)j0, (int32_t)j1,
                                        nch > 1 ? (int32_t)(slot + k) : -1, 0, 0});
                }
                i0 += ni;
                rest -= ni;
            }
            if (nch > 1) slot += nch;
        }
        OTOO_REQUIRE(slot <= INT32_MAX && P->items.size() <= (size_t)INT32_MAX, OTOO_EINVAL, "plan too large");
        P->partial_doubles = slot * 4 * (int64_t)ncm;
        std::vector<int64_t> cost(P->items.size());
        for (size_t i = 0; i < P->items.size(); ++i)
            cost[i] = (int64_t)P->items[i].ni * (P->items[i].j1 - P->items[i].j0);
        std::vector<int64_t> idx(P->items.size());
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
        std::vector<otoo_item> sorted(P->items.size());
        for (size_t i = 0; i < idx.size(); ++i) sorted[i] = P->items[idx[i]];
        P->items.swap(sorted);
        *out = P;
        return OTOO_OK;
    });
}

int otoo_plan_export(const otoo_plan* P, otoo_plan_info* info)
{
    OTOO_REQUIRE(P && info, OTOO_EINVAL, "otoo_plan_export: NULL argument");
    info->n_items = (int64_t)P->items.size();
    info->n_splits = (int64_t)P->splits.size();
    info->partial_doubles = P->partial_doubles;
    info->n_crit_max = P->n_crit_max;
    info->pad = 0;
    info->items = P->items.data();
    info->splits = P->splits.data();
    return OTOO_OK;
}

void otoo_plan_free(otoo_plan* P) { delete P; }

// Features of each group's list for the learned opening angle.
int otoo_group_features(const otoo_tree* t, const otoo_lists* L, float* feat)
{
    Range range_("otoo_group_features");
    OTOO_REQUIRE(t && L && feat, OTOO_EINVAL, "otoo_group_features: NULL argument");
    OTOO_REQUIRE(L->n_sys == 1 && L->n_part == t->n, OTOO_EINVAL, "features need the single-system lists of this tree");
    const int64_t G = (int64_t)L->groups.size();
    const int64_t n = t->n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t g = 0; g < G; ++g) {
        const otoo_group& og = L->groups[g];
        double blo[3], bhi[3];
        for (int a = 0; a < 3; ++a) blo[a] = bhi[a] = t->pos[3 * og.first + a];
        for (int64_t i = og.first + 1; i < og.first + og.count; ++i)
            for (int a = 0; a < 3; ++a) {
                blo[a] = std::min(blo[a], t->pos[3 * i + a]);
                bhi[a] = std::max(bhi[a], t->pos[3 * i + a]);
            }
        const double c[3] = {og.cx, og.cy, og.cz};
        double mincell = 1e3, mcell = 0, mall = 0;
        double hd = 0.5 * std::sqrt((bhi[0] - blo[0]) * (bhi[0] - blo[0]) + (bhi[1] - blo[1]) * (bhi[1] - blo[1]) +
                                    (bhi[2] - blo[2]) * (bhi[2] - blo[2]));
        const double eps = std::sqrt(og.eps2);
        hd = std::max(hd, eps * 1e-3);
        // the list's net pull at the group centre (every entry, softened) and
        // the cells' third-order spread terms B_2 b_max / d^5 (d: distance to
        // the group box), the size of the first term a quadrupole leaves out
        double anet[3] = {0, 0, 0}, trunc = 0;
        const int32_t* e = L->list.data() + og.list_off;
        for (int j = 0; j < og.n_cell + og.n_part; ++j) {
            const bool cell = j < og.n_cell;
            const int64_t k = cell ? e[j] - n : e[j];
            const double* x = cell ? &t->c_com[3 * k] : &t->pos[3 * k];
            const double m = cell ? t->c_mass[k] : (double)t->mass[k];
            double d2 = 0, r2 = 0, r[3];
            for (int a = 0; a < 3; ++a) {
                double d = 0;
                if (blo[a] - x[a] > d) d = blo[a] - x[a];
                if (x[a] - bhi[a] > d) d = x[a] - bhi[a];
                d2 += d * d;
                r[a] = x[a] - c[a];
                r2 += r[a] * r[a];
            }
            mall += m;
            const double rs2 = r2 + og.eps2;
            const double w = m / (rs2 * std::sqrt(rs2));
            for (int a = 0; a < 3; ++a) anet[a] += w * r[a];
            if (cell) {
                const double d = std::sqrt(d2);
                mincell = std::min(mincell, d / t->c_side[k]);
                mcell += m;
                const double dd = std::max(d, 1e-300);
                trunc += t->c_b2[k] * t->c_bmax[k] / (dd * dd * dd * dd * dd);
            }
        }
        const double an = std::sqrt(anet[0] * anet[0] + anet[1] * anet[1] + anet[2] * anet[2]);
        float* f = feat + 5 * g;
        f[0] = (float)std::log2((double)std::max(1, og.n_cell + og.n_part));
        f[1] = (float)std::log10(std::max(mincell, 1e-3));
        f[2] = (float)std::log10(hd / eps);
        f[3] = (float)(mall > 0 ? mcell / mall : 0.0);
        f[4] = (float)std::log10(std::max(trunc / std::max(an, 1e-300), 1e-12));
    }
    return OTOO_OK;
}

}  // extern "C"
