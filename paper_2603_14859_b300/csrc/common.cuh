// Shared host/device helpers of libvpetabc (error reporting, launch checks).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/vpetabc.h"

namespace vpet {

// Thread-local last-error text behind abc_last_error().
void set_error(const char* fmt, ...);
void clear_error();

// Process-wide count of kernels this library has launched (abc_launch_info).
void count_launch();

}  // namespace vpet

#define VPET_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            vpet::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return ABC_ERR_CUDA;                                                         \
        }                                                                                \
    } while (0)

#define VPET_ARG(cond, ...)                 \
    do {                                    \
        if (!(cond)) {                      \
            vpet::set_error(__VA_ARGS__);   \
            return ABC_ERR_ARG;             \
        }                                   \
    } while (0)

#define VPET_LAUNCH_CHECK()                                                              \
    do {                                                                                 \
        vpet::count_launch();                                                            \
        cudaError_t e_ = cudaGetLastError();                                             \
        if (e_ != cudaSuccess) {                                                         \
            vpet::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return ABC_ERR_CUDA;                                                         \
        }                                                                                \
    } while (0)

static inline int64_t vpet_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t vpet_round_up(int64_t a, int64_t b) { return vpet_ceil_div(a, b) * b; }
