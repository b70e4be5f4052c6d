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
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      cached = v;
    else
      return 148;
  }
  return cached;
}

int64_t& launch_counter() {
  static thread_local int64_t c = 0;
  return c;
}

}  // namespace ajd

extern "C" const char* jd_last_error(void) { return ajd::g_last_error.c_str(); }

extern "C" int jd_version(void) { return 100; }
