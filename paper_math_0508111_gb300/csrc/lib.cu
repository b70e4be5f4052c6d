#include <atomic>
// Library-wide helpers: error strings, version, device properties.
#include "common.cuh"

namespace ajd {

static thread_local std::string g_last_error;

void set_error_msg(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int sm_count() {
  // SMs of the current device, queried once per device (threads may ask
  // concurrently: relaxed atomics, every writer stores the same value)
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int v = cached[dev].load(std::memory_order_relaxed);
  if (v == 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 148;
    cached[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

int64_t& launch_counter() {
  static thread_local int64_t c = 0;
  return c;
}

}  // namespace ajd

extern "C" const char* jd_last_error(void) { return ajd::g_last_error.c_str(); }

extern "C" int jd_version(void) { return 100; }
