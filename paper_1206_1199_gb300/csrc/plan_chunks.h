// Particle chunks of the FP32 force kernel's work items, shared by the host
// plan (tree.cpp, otoo_make_plan) and the device plan (walk.cu,
// otoo_plan_count / otoo_plan_fill), so that both cut a group the same way.
//
// A work item of s targets runs on one warp with ib targets per lane: P =
// ceil(s / ib) lanes hold the targets and the warp's 32 lanes form nsub =
// 32 / P subsets that share the list's entries.  Lanes outside the subsets
// idle, so a group whose size does not fill the warp wastes lanes (a group of
// 26 at ib = 2: 13 lanes x 2 subsets, 6 lanes idle).  Cutting the group into
// items of sizes that fill the warp (16 + 10: 8 x 4 and 5 x 6 lanes) costs one
// more pass over the list (staging) but fewer idle lanes.  The table below
// holds, for every group size n, the last chunk of a cut of n that minimises
// a modelled warp time per list entry; the cut of n is last[n], then the cut
// of n - last[n].  Integer arithmetic only: both sides build identical
// tables.
#pragma once
#include <stdint.h>

#include "common.h"

#ifdef __CUDACC__
#define OTOO_PC_HD __host__ __device__ __forceinline__
#else
#define OTOO_PC_HD inline
#endif

namespace otoo {

struct ChunkTable {
    int32_t ib;                        // targets per lane the table was made for
    uint16_t last[kMaxGroup + 1];      // last chunk of the cut of n targets (last[0] = 0)
};

OTOO_PC_HD int32_t chunk_nsub(int32_t s, int32_t ib) { return 32 / ((s + ib - 1) / ib); }

// Modelled warp time of one item of s targets over a list of kChunkRefLen
// entries, in units of one warp-wide FP32 instruction: the pair steps (each
// lane takes ib targets against one entry per step, ~36 instructions per
// target for a quadrupole cell), the staging of every entry (kChunkStage
// per entry: the weight that gave the fastest step on GB300 among 1..4 for
// the Hernquist N = 2^23 lists), a fixed cost per item
// (ticket, item, group and target loads) and the pairwise merge of the nsub
// lane subsets (ceil(log2 nsub) rounds of shuffles and compensated adds).
constexpr int64_t kChunkRefLen = 4096;
constexpr int64_t kChunkStage = 4;
inline int64_t chunk_cost(int32_t s, int32_t ib)
{
    const int64_t nsub = chunk_nsub(s, ib);
    int64_t rounds = 0;
    while ((int64_t(1) << rounds) < nsub) ++rounds;
    return (kChunkRefLen + nsub - 1) / nsub * ib * 36 + kChunkStage * kChunkRefLen + 600 + rounds * 40;
}

// Fills t for ib >= 1 targets per lane (items of at most 32 * ib targets);
// ties go to the smaller last chunk.
inline void chunk_table_build(int32_t ib, ChunkTable& t)
{
    ib = ib < 1 ? 1 : ib;
    t.ib = ib;
    const int32_t smax = 32 * ib < kMaxGroup ? 32 * ib : kMaxGroup;
    int64_t cost[kMaxGroup + 1];
    int64_t cs[kMaxGroup + 1];
    for (int32_t s = 1; s <= smax; ++s) cs[s] = chunk_cost(s, ib);
    cost[0] = 0;
    t.last[0] = 0;
    for (int32_t m = 1; m <= kMaxGroup; ++m) {
        int64_t best = -1;
        int32_t arg = 1;
        for (int32_t s = 1; s <= m && s <= smax; ++s) {
            const int64_t c = cost[m - s] + cs[s];
            if (best < 0 || c < best) best = c, arg = s;
        }
        cost[m] = best;
        t.last[m] = (uint16_t)arg;
    }
}

// Number of chunks of n targets and the largest chunk.
OTOO_PC_HD int32_t chunk_count(const ChunkTable& t, int32_t n, int32_t* largest)
{
    int32_t c = 0, big = 0;
    while (n > 0) {
        const int32_t s = t.last[n];
        big = s > big ? s : big;
        n -= s;
        ++c;
    }
    if (largest) *largest = big;
    return c;
}

}  // namespace otoo
