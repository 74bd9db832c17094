// Exercises the host half of the C ABI (tree, groups and lists for the three
// acceptance rules, batch packing, plans, features, device arrays, exports,
// invalid inputs) on a seeded sample, for runs of the host library built with
// the address and undefined-behaviour sanitizers.  Exit status 0 when every
// call returned what it should.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "otoo.h"

namespace {

uint64_t g_state = 0x1206119912061199ull;
double uniform()  // xorshift64*, 53-bit uniform in [0, 1)
{
    g_state ^= g_state >> 12;
    g_state ^= g_state << 25;
    g_state ^= g_state >> 27;
    return (double)((g_state * 0x2545F4914F6CDD1Dull) >> 11) * (1.0 / 9007199254740992.0);
}

// Plummer-like cloud: radius from the inverse cumulative mass, isotropic.
void sample(int64_t n, std::vector<double>& pos, std::vector<float>& mass)
{
    pos.resize(3 * n);
    mass.assign(n, (float)(1.0 / (double)n));
    for (int64_t i = 0; i < n; ++i) {
        double x = uniform();
        if (x < 1e-6) x = 1e-6;
        const double r = 1.0 / std::sqrt(std::pow(x, -2.0 / 3.0) - 1.0 + 1e-12);
        const double ct = 2.0 * uniform() - 1.0, ph = 6.283185307179586 * uniform();
        const double st = std::sqrt(1.0 - ct * ct);
        pos[3 * i] = r * st * std::cos(ph);
        pos[3 * i + 1] = r * st * std::sin(ph);
        pos[3 * i + 2] = r * ct;
    }
}

int g_fail = 0;
void expect(bool ok, const char* what)
{
    if (!ok) {
        std::fprintf(stderr, "FAILED: %s (%s)\n", what, otoo_last_error());
        ++g_fail;
    }
}

}  // namespace

int main()
{
    const int64_t n = 20000;
    std::vector<double> pos;
    std::vector<float> mass;
    sample(n, pos, mass);
    otoo_params p = {};
    p.theta = 0.5;
    p.leaf_size = 8;
    p.n_crit = 64;
    p.use_quad = 1;
    p.mac = OTOO_MAC_THETA;
    p.eps = 0.01;
    otoo_tree* t = nullptr;
    expect(otoo_build_tree(pos.data(), mass.data(), n, &p, &t) == OTOO_OK, "build_tree");
    otoo_tree_view tv;
    expect(otoo_tree_export(t, &tv) == OTOO_OK && tv.n_part == n, "tree_export");

    // the three acceptance rules
    std::vector<float> h(n, 0.05f);
    otoo_lists* L[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) {
        otoo_params q = p;
        q.mac = k == 0 ? OTOO_MAC_THETA : k == 1 ? OTOO_MAC_SW : OTOO_MAC_SPH;
        q.delta = 1e-3;
        q.m_limit = 0.05;
        q.h_sph = k == 2 ? h.data() : nullptr;
        expect(otoo_make_groups_and_lists(t, &q, &L[k]) == OTOO_OK, "make_groups_and_lists");
        otoo_lists_view v;
        expect(otoo_lists_export(L[k], &v) == OTOO_OK && v.n_part == n, "lists_export");
    }
    // per-group angles, some groups skipped
    int64_t G = 0;
    expect(otoo_find_groups(t, 64, nullptr, nullptr, 0, &G) == OTOO_OK && G > 0, "find_groups count");
    std::vector<int32_t> first(G), count(G);
    expect(otoo_find_groups(t, 64, first.data(), count.data(), G, &G) == OTOO_OK, "find_groups");
    std::vector<float> tpg(G);
    for (int64_t g = 0; g < G; ++g) tpg[g] = g % 3 == 0 ? -1.f : 0.3f + 0.1f * (float)(g % 5);
    otoo_params q = p;
    q.theta_per_group = tpg.data();
    otoo_lists* Lt = nullptr;
    expect(otoo_make_groups_and_lists(t, &q, &Lt) == OTOO_OK, "per-group angles");

    // plans: every targets-per-lane choice, short and long list chunks
    for (int ib : {1, 2, 4})
        for (int split : {64, 300, 100000}) {
            otoo_tune tune;
            expect(otoo_default_tune(64, &tune) == OTOO_OK, "default_tune");
            tune.iblock = ib;
            tune.split = split;
            otoo_plan* P = nullptr;
            expect(otoo_make_plan(L[0], &tune, &P) == OTOO_OK, "make_plan");
            otoo_plan_info info;
            expect(otoo_plan_export(P, &info) == OTOO_OK && info.n_items > 0, "plan_export");
            otoo_plan_free(P);
        }

    // batch of two systems, features, device arrays
    const otoo_lists* two[2] = {L[0], Lt};
    otoo_lists* B = nullptr;
    expect(otoo_pack_batch(two, 2, &B) == OTOO_OK, "pack_batch");
    otoo_lists_view bv;
    expect(otoo_lists_export(B, &bv) == OTOO_OK && bv.n_part == 2 * n, "batch export");
    otoo_lists_view v0;
    otoo_lists_export(L[0], &v0);
    std::vector<float> feat((size_t)v0.n_groups * 8);
    expect(otoo_group_features(t, L[0], feat.data()) == OTOO_OK, "group_features");
    std::vector<otoo_src> src(n + tv.n_cell);
    std::vector<otoo_quad> quad(tv.n_cell);
    std::vector<otoo_wcell> cell(tv.n_cell);
    std::vector<otoo_wcell64> cell64(tv.n_cell);
    expect(otoo_tree_device_arrays(t, 1, &p, src.data(), quad.data(), cell.data(), cell64.data()) == OTOO_OK,
           "tree_device_arrays");

    // invalid inputs are refused with OTOO_EINVAL, nothing is written
    std::vector<double> bad = pos;
    bad[7] = NAN;
    otoo_tree* tb = nullptr;
    expect(otoo_build_tree(bad.data(), mass.data(), n, &p, &tb) == OTOO_EINVAL && tb == nullptr, "NaN position");
    otoo_params pb = p;
    pb.eps = 0.0;
    otoo_lists* lb = nullptr;
    expect(otoo_make_groups_and_lists(t, &pb, &lb) == OTOO_EINVAL && lb == nullptr, "eps = 0");
    pb = p;
    pb.n_crit = 5000;
    expect(otoo_make_groups_and_lists(t, &pb, &lb) == OTOO_EINVAL && lb == nullptr, "n_crit too large");
    expect(otoo_build_tree(pos.data(), mass.data(), 0, &p, &tb) == OTOO_EINVAL, "n = 0");

    otoo_lists_free(B);
    otoo_lists_free(Lt);
    for (otoo_lists* l : L) otoo_lists_free(l);
    otoo_tree_free(t);
    std::printf("host calls checked, %d failed\n", g_fail);
    return g_fail ? 1 : 0;
}
