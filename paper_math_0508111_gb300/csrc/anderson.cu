// The Anderson matrix of Eq. (1): disorder generation and the matrix-free
// 7-point stencil y = (A - shift I) x.
//
// Section 3.1 notes that the matrix-vector product can be coded directly with
// only the diagonal stored.  Here it is a z-marching stencil (see
// stencil_kernel below): every x value is read from HBM once per sweep and
// every y written once, 24 bytes per site in binary64 and 12 in binary32.
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

// Row-marching stencil.  A warp owns one x-segment of 32*V sites of a lattice
// row (fixed y) and walks a chunk of z-planes, keeping the segment's values at
// z-1, z and z+1 in registers; lane l holds sites seg*32V + l + 32v, so every
// load instruction of the warp is one contiguous, coalesced run.  The x+-1 and
// y+-1 neighbours are re-read through L1 (the eight warps of a CTA own eight
// consecutive rows), so each x value comes from HBM once per sweep.
constexpr int kWarps = 8;

template <typename T>
__device__ __forceinline__ T ldv(const T* __restrict__ p, int64_t i, bool ok) {
  return ok ? __ldg(p + i) : T(0);
}

template <typename T, int V>
__global__ void __launch_bounds__(32 * kWarps)
stencil_kernel(const T* __restrict__ eps, const T* __restrict__ xin, T* __restrict__ yout,
               int L, int nseg, int zchunk, T shift, T hop, int periodic_i, int64_t n) {
  const bool periodic = periodic_i != 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = blockIdx.x * kWarps + warp;
  if (w >= L * nseg) return;
  const int yy = w / nseg, seg = w - yy * nseg;
  const int z0 = blockIdx.y * zchunk;
  const int z1 = min(z0 + zchunk, L);
  const int64_t LL = (int64_t)L * L;
  const T* __restrict__ x = xin + (int64_t)blockIdx.z * n;
  T* __restrict__ y = yout + (int64_t)blockIdx.z * n;

  int xi[V], xl[V], xr[V];
  bool ok[V], okl[V], okr[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    xi[v] = seg * 32 * V + lane + 32 * v;
    ok[v] = xi[v] < L;
    xl[v] = xi[v] - 1;
    xr[v] = xi[v] + 1;
    okl[v] = ok[v] && (periodic || xl[v] >= 0);
    okr[v] = ok[v] && (periodic || xr[v] < L);
    if (xl[v] < 0) xl[v] += L;
    if (xr[v] >= L) xr[v] -= L;
  }
  int ym = yy - 1, yp = yy + 1;
  const bool okym = periodic || ym >= 0, okyp = periodic || yp < L;
  if (ym < 0) ym += L;
  if (yp >= L) yp -= L;

  // Software pipeline: x of planes z-1, z, z+1 are consumed at step z while
  // plane z+2 (x) and z+1 (eps) are in flight; planes further ahead are
  // prefetched into L2 so that the register loads hit L2 rather than HBM.
  auto wrapz = [&](int z, bool& okz) {
    okz = periodic || (z >= 0 && z < L);
    if (z < 0) z += L;
    if (z >= L) z -= L;
    return z;
  };
  T xm[V], xc[V], xp[V], xpp[V], ec[V], en[V];
  {
    bool o1, o2, o3;
    const int za = wrapz(z0 - 1, o1), zb = wrapz(z0 + 1, o2);
    const int64_t bm = (int64_t)za * LL + (int64_t)yy * L, b0 = (int64_t)z0 * LL + (int64_t)yy * L;
    const int64_t bp = (int64_t)zb * LL + (int64_t)yy * L;
    (void)o3;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      xm[v] = ldv(x, bm + xi[v], ok[v] && o1);
      xc[v] = ldv(x, b0 + xi[v], ok[v]);
      xp[v] = ldv(x, bp + xi[v], ok[v] && o2);
      ec[v] = ldv(eps, b0 + xi[v], ok[v]);
    }
  }
  constexpr int kPrefetch = 6;
  for (int z = z0; z < z1; ++z) {
    bool okpp, oke, okf;
    const int zpp = wrapz(z + 2, okpp);
    const int ze = wrapz(z + 1, oke);
    const int zf = wrapz(z + kPrefetch, okf);
    const int64_t row = (int64_t)z * LL + (int64_t)yy * L;
    const int64_t rowpp = (int64_t)zpp * LL + (int64_t)yy * L;
    const int64_t rowe = (int64_t)ze * LL + (int64_t)yy * L;
    const int64_t rowf = (int64_t)zf * LL + (int64_t)yy * L;
    const int64_t rowym = (int64_t)z * LL + (int64_t)ym * L;
    const int64_t rowyp = (int64_t)z * LL + (int64_t)yp * L;
    const bool more = z + 1 < z1;  // planes beyond this chunk are not needed
    T nb[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      xpp[v] = ldv(x, rowpp + xi[v], ok[v] && okpp && (z + 2 <= z1));
      en[v] = ldv(eps, rowe + xi[v], ok[v] && oke && more);
      if (ok[v] && okf && z + kPrefetch <= z1) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(x + rowf + xi[v]));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(eps + rowf + xi[v]));
      }
      nb[v] = ldv(x, row + xl[v], okl[v]) + ldv(x, row + xr[v], okr[v]);
      nb[v] += ldv(x, rowym + xi[v], ok[v] && okym) + ldv(x, rowyp + xi[v], ok[v] && okyp);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (ok[v]) y[row + xi[v]] = (ec[v] - shift) * xc[v] + hop * (nb[v] + xm[v] + xp[v]);
      xm[v] = xc[v];
      xc[v] = xp[v];
      xp[v] = xpp[v];
      ec[v] = en[v];
    }
  }
}

}  // namespace

template <typename T, int V>
static void launch_stencil(const T* eps, const T* x, T* y, int L, int m, T shift, T hop,
                           int periodic, int64_t n, cudaStream_t stream) {
  const int nseg = ceil_div(L, 32 * V);
  const int units = L * nseg;
  const int bx = ceil_div(units, kWarps);
  // enough CTAs to fill every SM several times over; z-chunks split the rest
  const int target = 8 * sm_count();
  int nchunk = ceil_div(target, (int64_t)bx * m);
  if (nchunk > L) nchunk = L;
  if (nchunk < 1) nchunk = 1;
  const int zchunk = ceil_div(L, nchunk);
  nchunk = ceil_div(L, zchunk);
  dim3 grid(bx, nchunk, m);
  stencil_kernel<T, V><<<grid, 32 * kWarps, 0, stream>>>(eps, x, y, L, nseg, zchunk, shift, hop,
                                                         periodic, n);
  count_launches();
}

template <typename T>
int stencil_apply(const anderson_s* h, T shift, const T* x, T* y, int m, cudaStream_t stream) {
  if (m == 0) return JD_OK;
  if (m > 65535) return fail(JD_EINVAL, "anderson_apply: at most 65535 vectors per call");
  const T* eps = nullptr;
  if constexpr (sizeof(T) == 8) eps = reinterpret_cast<const T*>(h->eps64);
  else eps = reinterpret_cast<const T*>(h->eps32);
  const int L = h->L, per = h->bc == JD_PERIODIC ? 1 : 0;
  const T hop = (T)h->hop;
  if (L <= 32) launch_stencil<T, 1>(eps, x, y, L, m, shift, hop, per, h->n, stream);
  else if (L <= 64) launch_stencil<T, 2>(eps, x, y, L, m, shift, hop, per, h->n, stream);
  else if (L <= 96) launch_stencil<T, 3>(eps, x, y, L, m, shift, hop, per, h->n, stream);
  else launch_stencil<T, 4>(eps, x, y, L, m, shift, hop, per, h->n, stream);
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

__global__ void narrow_kernel(const double* __restrict__ e64, float* __restrict__ e32, int64_t n) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
    e32[s] = (float)e64[s];
}

extern "C" int anderson_create_from_potential(int L, const double* eps_host, int bc, anderson_t* out) {
  if (!out || !eps_host) return fail(JD_EINVAL, "anderson_create_from_potential: NULL argument");
  *out = nullptr;
  if (bc != JD_PERIODIC && bc != JD_HARDWALL) return fail(JD_EINVAL, "anderson_create_from_potential: bad bc");
  if (bc == JD_PERIODIC && L < 3) return fail(JD_EINVAL, "anderson_create_from_potential: periodic lattice needs L >= 3");
  if (L < 1 || (int64_t)L * L * L >= (int64_t)1 << 31) return fail(JD_EINVAL, "anderson_create_from_potential: bad L");
  const int64_t n = (int64_t)L * L * L;
  double mx = 0.0;
  for (int64_t s = 0; s < n; ++s) {
    if (!std::isfinite(eps_host[s])) return fail(JD_EINVAL, "anderson_create_from_potential: non-finite eps");
    mx = std::max(mx, std::fabs(eps_host[s]));
  }
  anderson_s* h = new (std::nothrow) anderson_s();
  if (!h) return fail(JD_ENOMEM, "anderson_create_from_potential: host allocation failed");
  h->L = L;
  h->n = n;
  h->bc = bc;
  h->max_abs_eps = mx;
  cudaGetDevice(&h->device);
  cudaError_t e = cudaMalloc(&h->eps64, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->eps32, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(h->eps64, eps_host, n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 16 * sm_count());
    narrow_kernel<<<blocks, 256>>>(h->eps64, h->eps32, n);
    count_launches();
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    anderson_destroy(h);
    return fail(e == cudaErrorMemoryAllocation ? JD_ENOMEM : JD_EDEVICE, "anderson_create_from_potential: %s",
                cudaGetErrorString(e));
  }
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
