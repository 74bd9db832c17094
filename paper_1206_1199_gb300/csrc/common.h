// Internal helpers shared by the host and device translation units of libotoo.
#pragma once
#include <cstdarg>
#include <cstdio>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "otoo.h"

namespace otoo {

// Records the message of the last error on this thread; returns code.
int set_error(int code, const char* fmt, ...);

// Largest group the device kernels accept (threads * particles per thread).
constexpr int kMaxGroup = 1024;

// An NVTX range over one C entry point (tree, walk, plan, force, ...), for
// profilers that show or filter by ranges; next to free when no tool listens.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

// Enqueues the float-pair split of the FP32 form on a CUDA stream: out[2 s] =
// (x, y, z rounded to FP32, m), out[2 s + 1] = (the rounding remainders, 0)
// for the n sources (force.cu).  Returns OTOO_OK or OTOO_ECUDA.
int enqueue_split(const otoo_src* src, float* out, int64_t n, void* stream);

}  // namespace otoo

#define OTOO_REQUIRE(cond, code, ...)                      \
    do {                                                   \
        if (!(cond)) return ::otoo::set_error(code, __VA_ARGS__); \
    } while (0)
