// The Anderson matrix of Eq. (1): disorder generation and the matrix-free
// 7-point stencil y = (A - shift I) x.
//
// Section 3.1 notes that the matrix-vector product can be coded directly with
// only the diagonal stored.  Here the product is a z-marching stencil: each
// CTA owns a TX x TY column of the lattice and walks a chunk of z-planes,
// keeping the (z-1, z, z+1) values of its column in registers and staging
// the current plane (plus a one-site halo, wrapped for periodic boundaries)
// in shared memory.  Every x value is read from HBM once per sweep, every
// y written once: 24 bytes per site in binary64, 12 in binary32.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "anderson_impl.cuh"

namespace ajd {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kMul1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kMul2 = 0x94D049BB133111EBull;

// The idx-th output of SplitMix64 seeded with `seed` (counter form: the
// idx-th state is seed + (idx + 1) * gamma).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1ull) * kGamma;
  z = (z ^ (z >> 30)) * kMul1;
  z = (z ^ (z >> 27)) * kMul2;
  return z ^ (z >> 31);
}

// eps_s = W (u_s - 1/2), u_s = top 53 bits of output s times 2^-53
// (box distribution on [-W/2, W/2), Section 3).
__global__ void potential_kernel(double* __restrict__ eps64, float* __restrict__ eps32,
                                 int64_t n, uint64_t seed, double W) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = splitmix64_at(seed, (uint64_t)s);
    double u = __dmul_rn((double)(z >> 11), 0x1.0p-53);
    double e = __dmul_rn(W, __dsub_rn(u, 0.5));
    eps64[s] = e;
    eps32[s] = (float)e;
  }
}

// max_s |eps_s| by an atomic max on the IEEE bit pattern (valid because all
// compared values are non-negative).
__global__ void max_abs_kernel(const double* __restrict__ v, int64_t n,
                               unsigned long long* out) {
  double m = 0.0;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(v[s]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

constexpr int TX = 32;  // tile width (x, contiguous in memory)
constexpr int TY = 8;   // tile height (y)

template <typename T>
__device__ __forceinline__ T load_site(const T* __restrict__ x, int L, int64_t LL,
                                       int wx, int wy, int z, bool inside_xy,
                                       bool periodic) {
  if (periodic) {
    z = (z < 0) ? z + L : (z >= L ? z - L : z);
  } else if (z < 0 || z >= L || !inside_xy) {
    return T(0);
  }
  return __ldg(x + (int64_t)z * LL + (int64_t)wy * L + wx);
}

// y = (eps - shift) x + hop * (sum of the six neighbours), one vector per
// blockIdx.z.  Tiles of TX x TY sites in (x, y); blockIdx.y picks a chunk of
// `zchunk` planes.
template <typename T>
__global__ void __launch_bounds__(TX * TY)
stencil_kernel(const T* __restrict__ eps, const T* __restrict__ xin, T* __restrict__ yout,
               int L, int ntx, int zchunk, T shift, T hop, int periodic_i, int64_t n) {
  __shared__ T tile[TY + 2][TX + 2];
  const bool periodic = periodic_i != 0;
  const int64_t LL = (int64_t)L * L;
  const T* __restrict__ x = xin + (int64_t)blockIdx.z * n;
  T* __restrict__ y = yout + (int64_t)blockIdx.z * n;
  const int tx0 = (blockIdx.x % ntx) * TX;
  const int ty0 = (blockIdx.x / ntx) * TY;
  const int z0 = blockIdx.y * zchunk;
  const int z1 = min(z0 + zchunk, L);
  if (z0 >= L) return;
  const int lx = threadIdx.x, ly = threadIdx.y;
  const int gx = tx0 + lx, gy = ty0 + ly;
  const bool own = gx < L && gy < L;
  // coordinates this thread's register column holds (wrapped for periodic,
  // zero outside for hard walls)
  const int wx = periodic ? gx % L : gx;
  const int wy = periodic ? gy % L : gy;
  const bool in_xy = periodic || own;

  // halo perimeter: cells of the (TY+2) x (TX+2) frame, filled by the first
  // threads of the block
  const int tid = ly * TX + lx;
  constexpr int kPerim = 2 * (TX + 2) + 2 * TY;
  int hr = 0, hc = 0;
  if (tid < kPerim) {
    if (tid < TX + 2) { hr = 0; hc = tid; }
    else if (tid < 2 * (TX + 2)) { hr = TY + 1; hc = tid - (TX + 2); }
    else { int k = tid - 2 * (TX + 2); hr = 1 + (k >> 1); hc = (k & 1) ? TX + 1 : 0; }
  }
  int hx = tx0 + hc - 1, hy = ty0 + hr - 1;
  bool h_in = true;
  if (periodic) {
    hx = (hx + L) % L;
    hy = (hy + L) % L;
  } else {
    h_in = hx >= 0 && hx < L && hy >= 0 && hy < L;
  }

  T prev = load_site(x, L, LL, wx, wy, z0 - 1, in_xy, periodic);
  T cur = load_site(x, L, LL, wx, wy, z0, in_xy, periodic);
  T next;
  for (int z = z0; z < z1; ++z) {
    next = load_site(x, L, LL, wx, wy, z + 1, in_xy, periodic);
    tile[ly + 1][lx + 1] = cur;
    if (tid < kPerim) tile[hr][hc] = load_site(x, L, LL, hx, hy, z, h_in, periodic);
    __syncthreads();
    if (own) {
      const int64_t s = (int64_t)z * LL + (int64_t)gy * L + gx;
      T nb = tile[ly + 1][lx] + tile[ly + 1][lx + 2];
      nb += tile[ly][lx + 1] + tile[ly + 2][lx + 1];
      nb += prev + next;
      y[s] = (__ldg(eps + s) - shift) * cur + hop * nb;
    }
    __syncthreads();
    prev = cur;
    cur = next;
  }
}

}  // namespace

template <typename T>
int stencil_apply(const anderson_s* h, T shift, const T* x, T* y, int m, cudaStream_t stream) {
  if (m == 0) return JD_OK;
  const int L = h->L;
  const int ntx = ceil_div(L, TX), nty = ceil_div(L, TY);
  const int tiles = ntx * nty;
  const int target = 8 * sm_count();
  int nchunk = ceil_div(target, tiles);
  if (nchunk > L) nchunk = L;
  if (nchunk < 1) nchunk = 1;
  const int zchunk = ceil_div(L, nchunk);
  nchunk = ceil_div(L, zchunk);
  if (m > 65535) return fail(JD_EINVAL, "anderson_apply: at most 65535 vectors per call");
  dim3 grid(tiles, nchunk, m), block(TX, TY);
  const T* eps = nullptr;
  if constexpr (sizeof(T) == 8) eps = reinterpret_cast<const T*>(h->eps64);
  else eps = reinterpret_cast<const T*>(h->eps32);
  stencil_kernel<T><<<grid, block, 0, stream>>>(eps, x, y, L, ntx, zchunk, shift, (T)h->hop,
                                                h->bc == JD_PERIODIC ? 1 : 0, h->n);
  AJD_CHECK_LAUNCH();
  return JD_OK;
}

template int stencil_apply<double>(const anderson_s*, double, const double*, double*, int, cudaStream_t);
template int stencil_apply<float>(const anderson_s*, float, const float*, float*, int, cudaStream_t);

}  // namespace ajd

using namespace ajd;

extern "C" int anderson_create(int L, double W, uint64_t seed, int bc, anderson_t* out) {
  if (!out) return fail(JD_EINVAL, "anderson_create: out is NULL");
  *out = nullptr;
  if (bc != JD_PERIODIC && bc != JD_HARDWALL) return fail(JD_EINVAL, "anderson_create: bc must be JD_PERIODIC or JD_HARDWALL");
  if (bc == JD_PERIODIC && L < 3) return fail(JD_EINVAL, "anderson_create: periodic lattice needs L >= 3 (got %d)", L);
  if (L < 1) return fail(JD_EINVAL, "anderson_create: L must be >= 1 (got %d)", L);
  if ((int64_t)L * L * L >= (int64_t)1 << 31) return fail(JD_EINVAL, "anderson_create: L^3 must be < 2^31");
  if (!(W >= 0.0) || !std::isfinite(W)) return fail(JD_EINVAL, "anderson_create: W must be finite and >= 0");
  anderson_s* h = new (std::nothrow) anderson_s();
  if (!h) return fail(JD_ENOMEM, "anderson_create: host allocation failed");
  h->L = L;
  h->n = (int64_t)L * L * L;
  h->W = W;
  h->seed = seed;
  h->bc = bc;
  cudaGetDevice(&h->device);
  unsigned long long* dmax = nullptr;
  cudaError_t e = cudaMalloc(&h->eps64, h->n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->eps32, h->n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dmax, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(h->eps64);
    cudaFree(h->eps32);
    cudaFree(dmax);
    delete h;
    return fail(e == cudaErrorMemoryAllocation ? JD_ENOMEM : JD_EDEVICE,
                "anderson_create: %s", cudaGetErrorString(e));
  }
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((h->n + threads - 1) / threads, 16 * sm_count());
  cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), 0);
  potential_kernel<<<blocks, threads>>>(h->eps64, h->eps32, h->n, seed, W);
  max_abs_kernel<<<blocks, threads>>>(h->eps64, h->n, dmax);
  unsigned long long bits = 0;
  e = cudaMemcpy(&bits, dmax, sizeof(bits), cudaMemcpyDeviceToHost);
  cudaFree(dmax);
  if (e != cudaSuccess) {
    anderson_destroy(h);
    return fail(JD_EDEVICE, "anderson_create: %s", cudaGetErrorString(e));
  }
  std::memcpy(&h->max_abs_eps, &bits, sizeof(double));
  *out = h;
  return JD_OK;
}

extern "C" int anderson_destroy(anderson_t h) {
  if (!h) return JD_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(h->device);
  cudaFree(h->eps64);
  cudaFree(h->eps32);
  cudaSetDevice(dev);
  delete h;
  return JD_OK;
}

extern "C" int anderson_size(anderson_t h, int64_t* n) {
  if (!h || !n) return fail(JD_EINVAL, "anderson_size: NULL argument");
  *n = h->n;
  return JD_OK;
}

extern "C" int anderson_potential(anderson_t h, double* eps_host) {
  if (!h || !eps_host) return fail(JD_EINVAL, "anderson_potential: NULL argument");
  AJD_CUDA(cudaMemcpy(eps_host, h->eps64, h->n * sizeof(double), cudaMemcpyDeviceToHost));
  return JD_OK;
}

extern "C" int anderson_norm(anderson_t h, double* norm) {
  if (!h || !norm) return fail(JD_EINVAL, "anderson_norm: NULL argument");
  *norm = 6.0 + h->max_abs_eps;
  return JD_OK;
}

extern "C" int anderson_apply(anderson_t h, double shift, const void* x, void* y, int m,
                              int precision, void* stream) {
  if (!h) return fail(JD_EINVAL, "anderson_apply: NULL handle");
  if (m < 0) return fail(JD_EINVAL, "anderson_apply: m < 0");
  if (m == 0) return JD_OK;
  if (!x || !y) return fail(JD_EINVAL, "anderson_apply: NULL vector");
  if (x == y) return fail(JD_EINVAL, "anderson_apply: x and y must not overlap");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == JD_FP64)
    return stencil_apply<double>(h, shift, static_cast<const double*>(x), static_cast<double*>(y), m, s);
  if (precision == JD_FP32)
    return stencil_apply<float>(h, (float)shift, static_cast<const float*>(x), static_cast<float*>(y), m, s);
  return fail(JD_EINVAL, "anderson_apply: unknown precision %d", precision);
}
