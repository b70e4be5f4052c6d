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

// Off-diagonal model (Section 7): bond (s, d) from site s to its +d
// neighbour gets t = width (u_{3s+d} - 1/2), u from the same SplitMix64
// stream as the potential; hard walls zero the bonds that leave the cube.
__global__ void bond_kernel(double* __restrict__ b64, float* __restrict__ b32, int L, int64_t n, uint64_t seed,
                            double width, int periodic) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / 3;
    const int d = (int)(i - 3 * s);
    const int64_t c = d == 0 ? s % L : d == 1 ? (s / L) % L : s / ((int64_t)L * L);
    double t = 0.0;
    if (periodic || c < L - 1) {
      const uint64_t z = splitmix64_at(seed, (uint64_t)i);
      const double u = __dmul_rn((double)(z >> 11), 0x1.0p-53);
      t = __dmul_rn(width, __dsub_rn(u, 0.5));
    }
    b64[i] = t;
    b32[i] = (float)t;
  }
}

__global__ void fill_kernel(double* __restrict__ e64, float* __restrict__ e32, int64_t n, double v) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    e64[s] = v;
    e32[s] = (float)v;
  }
}

// y = (A - shift I) x for the off-diagonal model: one thread per site, the
// six neighbours weighted by their bonds (own +d bonds at [3s + d], the -d
// bonds stored at the neighbour).  Neighbour values and bonds are reused
// through the caches.
template <typename T>
__global__ void stencil_bond_kernel(const T* __restrict__ diag, const T* __restrict__ bond, const T* __restrict__ xin,
                                    T* __restrict__ yout, int L, T shift, int periodic, int64_t n) {
  const T* __restrict__ x = xin + (int64_t)blockIdx.y * n;
  T* __restrict__ y = yout + (int64_t)blockIdx.y * n;
  const int64_t LL = (int64_t)L * L;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c[3] = {s % L, (s / L) % L, s / LL};
    const int64_t step[3] = {1, L, LL};
    T acc = (__ldg(diag + s) - shift) * __ldg(x + s);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // +d neighbour through the own bond
      if (c[d] < L - 1) acc += __ldg(bond + 3 * s + d) * __ldg(x + s + step[d]);
      else if (periodic) acc += __ldg(bond + 3 * s + d) * __ldg(x + s - (L - 1) * step[d]);
      // -d neighbour through its bond
      if (c[d] > 0) acc += __ldg(bond + 3 * (s - step[d]) + d) * __ldg(x + s - step[d]);
      else if (periodic) {
        const int64_t sn = s + (L - 1) * step[d];
        acc += __ldg(bond + 3 * sn + d) * __ldg(x + sn);
      }
    }
    y[s] = acc;
  }
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

// Plane-tile stencil for rows whose length in bytes is a multiple of 16 (L a
// multiple of 4 in binary32, of 2 in binary64) and 16-byte aligned vectors.
// A CTA of 8 warps owns 8 consecutive y-rows of one x-segment (32 lanes x
// VW sites, VW = 16 B / element) and walks a chunk of z-planes.  Per step:
// every lane loads its VW sites with one 16-byte load (plane z+2 and the
// potential of plane z+1 are in flight while plane z is computed); the
// segment's 8 rows and the two halo rows y0-1, y0+8 pass through a
// shared-memory plane tile for the y-neighbours; x-neighbours come from the
// neighbouring lanes by shuffles (global loads only at segment ends); z-
// neighbours stay in registers.  DRAM traffic per site: x once (plus the
// halo rows, 2/8, mostly L2 hits), the potential once, y once.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <typename T>
__device__ __forceinline__ void vload(const T* __restrict__ p, bool ok, T (&v)[Vec16<T>::n]) {
  using V = typename Vec16<T>::type;
  if (ok) {
    const V q = __ldg(reinterpret_cast<const V*>(p));
    const T* e = reinterpret_cast<const T*>(&q);
#pragma unroll
    for (int i = 0; i < Vec16<T>::n; ++i) v[i] = e[i];
  } else {
#pragma unroll
    for (int i = 0; i < Vec16<T>::n; ++i) v[i] = T(0);
  }
}

constexpr int kTileRows = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kTileRows)
stencil_tile_kernel(const T* __restrict__ eps, const T* __restrict__ xin, T* __restrict__ yout, int L, int nseg,
                    int zchunk, T shift, T hop, int periodic_i, int64_t n) {
  constexpr int VW = Vec16<T>::n;
  using V = typename Vec16<T>::type;
  __shared__ V tile[kTileRows + 2][32];
  const bool periodic = periodic_i != 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int seg = blockIdx.x % nseg, ytile = blockIdx.x / nseg;
  const int y = ytile * kTileRows + warp;
  const int xs = seg * 32 * VW + VW * lane;  // first site of this lane
  const bool lane_ok = xs < L;               // L is a multiple of VW
  const bool own_ok = lane_ok && y < L;      // rows this warp writes
  // rows of the last tile beyond L hold the wrapped rows (periodic) or zeros,
  // so that row L-1 finds its y+1 neighbour in the tile
  const int yl = y < L ? y : (periodic ? y - L : -1);
  const bool load_ok = lane_ok && yl >= 0;
  const int z0 = blockIdx.y * zchunk;
  const int z1 = min(z0 + zchunk, L);
  const int64_t LL = (int64_t)L * L;
  const T* __restrict__ x = xin + (int64_t)blockIdx.z * n;
  T* __restrict__ yo = yout + (int64_t)blockIdx.z * n;
  // halo rows of this tile (loaded by warps 0 and kTileRows-1)
  int yh = -1;
  bool halo_ok = false;
  if (warp == 0 || warp == kTileRows - 1) {
    yh = warp == 0 ? ytile * kTileRows - 1 : ytile * kTileRows + kTileRows;
    halo_ok = periodic || (yh >= 0 && yh < L);
    if (yh < 0) yh += L;
    if (yh >= L) yh -= L;
    halo_ok = halo_ok && lane_ok && yh < L;
  }
  auto plane_ok = [&](int z, int& zz) {
    zz = z;
    if (zz < 0) zz += L;
    if (zz >= L) zz -= L;
    return periodic || (z >= 0 && z < L);
  };
  const bool last_lane = xs + VW >= L || lane == 31;  // its right neighbour lies in another segment
  T xm[VW], xc[VW], xp[VW], xq[VW], ec[VW], en[VW], hc[VW], hn[VW];
  {
    int za, zb;
    const bool oa = plane_ok(z0 - 1, za), ob = plane_ok(z0 + 1, zb);
    const int64_t r = (int64_t)(load_ok ? yl : 0) * L + xs;
    vload(x + (int64_t)za * LL + r, load_ok && oa, xm);
    vload(x + (int64_t)z0 * LL + r, load_ok, xc);
    vload(x + (int64_t)zb * LL + r, load_ok && ob, xp);
    vload(eps + (int64_t)z0 * LL + r, own_ok, ec);
    vload(x + (int64_t)z0 * LL + (int64_t)yh * L + xs, halo_ok, hc);
  }
  for (int z = z0; z < z1; ++z) {
    // loads for the next steps: x of plane z+2, eps and halo of plane z+1
    int zq, ze;
    const bool oq = plane_ok(z + 2, zq), oe = plane_ok(z + 1, ze);
    const bool more = z + 1 < z1;
    const int64_t r = (int64_t)(load_ok ? yl : 0) * L + xs;
    vload(x + (int64_t)zq * LL + r, load_ok && oq && z + 2 <= z1, xq);
    vload(eps + (int64_t)ze * LL + r, own_ok && more, en);
    vload(x + (int64_t)ze * LL + (int64_t)yh * L + xs, halo_ok && more, hn);
    // x-neighbours at the segment ends (global, usually L1/L2 hits)
    const int64_t row = (int64_t)z * LL + (int64_t)y * L;
    T left_g = T(0), right_g = T(0);
    if (own_ok && lane == 0) {
      const int xl = xs - 1;
      if (xl >= 0) left_g = x[row + xl];
      else if (periodic) left_g = x[row + L - 1];
    }
    if (own_ok && last_lane) {
      const int xr = xs + VW;
      if (xr < L) right_g = x[row + xr];
      else if (periodic) right_g = x[row];
    }
    // y-neighbours through the plane tile
    __syncthreads();  // the previous step's readers are done
    {
      V v;
      T* e = reinterpret_cast<T*>(&v);
#pragma unroll
      for (int i = 0; i < VW; ++i) e[i] = xc[i];
      tile[warp + 1][lane] = v;
      if (warp == 0 || warp == kTileRows - 1) {
#pragma unroll
        for (int i = 0; i < VW; ++i) e[i] = hc[i];
        tile[warp == 0 ? 0 : kTileRows + 1][lane] = v;
      }
    }
    __syncthreads();
    const V vm = tile[warp][lane], vp = tile[warp + 2][lane];
    const T* ym = reinterpret_cast<const T*>(&vm);
    const T* yp = reinterpret_cast<const T*>(&vp);
    // rows y-1 / y+1 outside a hard wall are zero
    const bool okym = periodic || y - 1 >= 0;
    const bool okyp = periodic || y + 1 < L;
    T left = __shfl_up_sync(0xffffffffu, xc[VW - 1], 1);
    T right = __shfl_down_sync(0xffffffffu, xc[0], 1);
    if (lane == 0) left = left_g;
    if (last_lane) right = right_g;
    if (own_ok) {
      T out[VW];
#pragma unroll
      for (int i = 0; i < VW; ++i) {
        const T l = i == 0 ? left : xc[i - 1];
        const T rr = i == VW - 1 ? right : xc[i + 1];
        const T nb = (l + rr) + ((okym ? ym[i] : T(0)) + (okyp ? yp[i] : T(0))) + (xm[i] + xp[i]);
        out[i] = (ec[i] - shift) * xc[i] + hop * nb;
      }
      V o;
      T* oe = reinterpret_cast<T*>(&o);
#pragma unroll
      for (int i = 0; i < VW; ++i) oe[i] = out[i];
      *reinterpret_cast<V*>(yo + row + xs) = o;
    }
#pragma unroll
    for (int i = 0; i < VW; ++i) {
      xm[i] = xc[i];
      xc[i] = xp[i];
      xp[i] = xq[i];
      ec[i] = en[i];
      hc[i] = hn[i];
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
static void launch_stencil_tile(const T* eps, const T* x, T* y, int L, int m, T shift, T hop, int periodic,
                                int64_t n, cudaStream_t stream) {
  constexpr int VW = Vec16<T>::n;
  const int nseg = ceil_div(L, 32 * VW);
  const int bx = nseg * ceil_div(L, kTileRows);
  // z-chunks: about eight CTAs per SM (measured at L = 256 against 2, 4 and
  // 16 per SM and 4- or 16-row tiles: 4.4 TB/s versus 2.7-4.2), each chunk
  // at least 8 planes
  const int target = 8 * sm_count();
  int nchunk = ceil_div(target, (int64_t)bx * m);
  nchunk = std::max(1, std::min(nchunk, std::max(1, L / 8)));
  const int zchunk = ceil_div(L, nchunk);
  nchunk = ceil_div(L, zchunk);
  dim3 grid(bx, nchunk, m);
  stencil_tile_kernel<T><<<grid, 32 * kTileRows, 0, stream>>>(eps, x, y, L, nseg, zchunk, shift, hop, periodic, n);
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
  if (h->bond64) {  // off-diagonal model
    const T* bond = nullptr;
    if constexpr (sizeof(T) == 8) bond = reinterpret_cast<const T*>(h->bond64);
    else bond = reinterpret_cast<const T*>(h->bond32);
    const int blocks = (int)std::min<int64_t>((h->n + 255) / 256, 16 * sm_count());
    stencil_bond_kernel<T><<<dim3(blocks, m), 256, 0, stream>>>(eps, bond, x, y, L, shift, per, h->n);
    count_launches();
    AJD_CHECK_LAUNCH();
    return JD_OK;
  }
  const T hop = (T)h->hop;
  // 16-byte rows and 16-byte aligned vectors: the plane-tile kernel
  constexpr int VW = Vec16<T>::n;
  const bool aligned = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) |
                         reinterpret_cast<uintptr_t>(eps)) % 16) == 0;
  if (L % VW == 0 && aligned && L >= 16) {
    launch_stencil_tile<T>(eps, x, y, L, m, shift, hop, per, h->n, stream);
    AJD_CHECK_LAUNCH();
    return JD_OK;
  }
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

extern "C" int anderson_create_offdiag(int L, double diag, double width, uint64_t seed, int bc, anderson_t* out) {
  if (!out) return fail(JD_EINVAL, "anderson_create_offdiag: out is NULL");
  *out = nullptr;
  if (bc != JD_PERIODIC && bc != JD_HARDWALL) return fail(JD_EINVAL, "anderson_create_offdiag: bad bc");
  if (bc == JD_PERIODIC && L < 3) return fail(JD_EINVAL, "anderson_create_offdiag: periodic lattice needs L >= 3");
  if (L < 1 || (int64_t)L * L * L >= ((int64_t)1 << 31) / 3) return fail(JD_EINVAL, "anderson_create_offdiag: bad L");
  if (!std::isfinite(diag) || !(width >= 0.0) || !std::isfinite(width))
    return fail(JD_EINVAL, "anderson_create_offdiag: diag must be finite and width finite and >= 0");
  anderson_s* h = new (std::nothrow) anderson_s();
  if (!h) return fail(JD_ENOMEM, "anderson_create_offdiag: host allocation failed");
  h->L = L;
  h->n = (int64_t)L * L * L;
  h->W = width;
  h->seed = seed;
  h->bc = bc;
  h->max_abs_eps = std::fabs(diag);
  cudaGetDevice(&h->device);
  const int64_t n = h->n;
  unsigned long long* dmax = nullptr;
  cudaError_t e = cudaMalloc(&h->eps64, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->eps32, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->bond64, 3 * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->bond32, 3 * n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&dmax, sizeof(unsigned long long));
  if (e == cudaSuccess) {
    const int blocks = (int)std::min<int64_t>((3 * n + 255) / 256, 16 * sm_count());
    fill_kernel<<<blocks, 256>>>(h->eps64, h->eps32, n, diag);
    bond_kernel<<<blocks, 256>>>(h->bond64, h->bond32, L, n, seed, width, bc == JD_PERIODIC ? 1 : 0);
    cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), 0);
    max_abs_kernel<<<blocks, 256>>>(h->bond64, 3 * n, dmax);
    count_launches(3);
    unsigned long long bits = 0;
    e = cudaMemcpy(&bits, dmax, sizeof(bits), cudaMemcpyDeviceToHost);
    std::memcpy(&h->max_abs_bond, &bits, sizeof(double));
  }
  cudaFree(dmax);
  if (e != cudaSuccess) {
    anderson_destroy(h);
    return fail(e == cudaErrorMemoryAllocation ? JD_ENOMEM : JD_EDEVICE, "anderson_create_offdiag: %s",
                cudaGetErrorString(e));
  }
  *out = h;
  return JD_OK;
}

extern "C" int anderson_bonds(anderson_t h, double* bonds_host) {
  if (!h || !bonds_host) return fail(JD_EINVAL, "anderson_bonds: NULL argument");
  if (!h->bond64) return fail(JD_EINVAL, "anderson_bonds: the lattice has constant hopping (Eq. (1))");
  AJD_CUDA(cudaMemcpy(bonds_host, h->bond64, 3 * h->n * sizeof(double), cudaMemcpyDeviceToHost));
  return JD_OK;
}

extern "C" int anderson_destroy(anderson_t h) {
  if (!h) return JD_OK;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(h->device);
  cudaFree(h->eps64);
  cudaFree(h->eps32);
  cudaFree(h->bond64);
  cudaFree(h->bond32);
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
  *norm = h->norm_bound();
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
