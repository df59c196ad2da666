// Host-side plumbing of the C ABI: per-thread error messages, CUDA error translation, device queries.
#include <cstdarg>
#include <cstdio>
#include <string>

#include "ms_device.cuh"

namespace {
thread_local std::string g_last_error;
}

namespace ms {

ms_status set_error(ms_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

ms_status cuda_status(cudaError_t e, const char* what)
{
    return set_error(MS_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

int num_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return 148;
    return sms;
}

}  // namespace ms

extern "C" const char* ms_last_error(void) { return g_last_error.c_str(); }

extern "C" int ms_version(void) { return 10000; }
