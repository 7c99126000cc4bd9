// Error reporting and launch accounting for libleg.
#include <stdarg.h>

#include "common.cuh"

namespace leg {

static thread_local char g_err[512] = "";
static thread_local int64_t g_launches = 0;

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

void count_launch(int n) { g_launches += n; }

}  // namespace leg

extern "C" const char* le_last_error(void) { return leg::g_err; }
extern "C" int64_t le_launch_count(void) { return leg::g_launches; }
extern "C" void le_reset_launch_count(void) { leg::g_launches = 0; }
