// Internal helpers shared by the host and device translation units of libotoo.
#pragma once
#include <cstdarg>
#include <cstdio>
#include <string>

#include "otoo.h"

namespace otoo {

// Records the message of the last error on this thread; returns code.
int set_error(int code, const char* fmt, ...);

// Largest group the device kernels accept (threads * particles per thread).
constexpr int kMaxGroup = 1024;

}  // namespace otoo

#define OTOO_REQUIRE(cond, code, ...)                      \
    do {                                                   \
        if (!(cond)) return ::otoo::set_error(code, __VA_ARGS__); \
    } while (0)
