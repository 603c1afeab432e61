// Error reporting for the C ABI (thread-local last-error text).
#include <stdarg.h>

#include <atomic>

#include "common.cuh"

namespace {
thread_local char g_err[512] = {0};
std::atomic<long long> g_launches{0};
}

namespace vpet {

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

long long launches() { return g_launches.load(std::memory_order_relaxed); }

}  // namespace vpet

extern "C" const char* abc_last_error(void) { return g_err; }
