// olb_ade.cu -- advection-diffusion BGK on D2Q5 / D3Q7 (section "Advection--
// Diffusion Equation"): a passive scalar C transported by a prescribed velocity v,
//   g*_i = g_i - omega (g_i - g^eq_i),   g^eq_i = w_i C (1 + c_i . v / cs2),
//   C = sum_i g_i,  diffusivity mu = cs2 (tau - 1/2),
// then periodic streaming g_i(x + c_i, t + 1) = g*_i(x, t).  The guide prints the
// first-order equilibrium and names the D2Q5 / D3Q7 descriptors without their
// tables: rest velocity first, the face velocities in the D2Q9 order, weights from
// sum w = 1 and sum w c_a c_b = cs2 delta_ab (cs2 = 1/3 and 1/4).
//
// One fused kernel per step, one cell per thread, push form on the canonical
// (pre-collision) state: the thread loads its own q values (coalesced), collides
// and stores each post-collision value at x + c_i of the other buffer (coalesced up
// to a one-element shift).  7 x 2 stored values per cell update.
//
// Boundaries (section "Advection--Diffusion Equation" names a constant-temperature
// boundary without its scheme; read as anti-bounce-back, the oracle's reading): a
// link of a bulk cell x that hits a no-flux wall cell, or leaves the domain along a
// non-periodic axis, bounces back, g_opp(i)(x) = g*_i(x); one that hits a Dirichlet
// cell of value C_w reflects with the opposite sign, g_opp(i)(x) = -g*_i(x) + 2 w_i C_w,
// which holds C_w at the link's midpoint.  Non-bulk cells keep their values.  A
// host-made mask per cell marks the links that need this, so bulk cells away from
// walls take no extra load beyond the mask.
#include <cuda_runtime.h>

#include <cstdint>

#include "olb_internal.h"

namespace olb {
namespace {

struct D2Q5 {
  static constexpr int Q = 5, DIM = 2;
  __device__ static constexpr int c(int i, int a) {
    constexpr int t[5][3] = {{0, 0, 0}, {-1, 0, 0}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}};
    return t[i][a];
  }
  __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
  static constexpr double cs2 = 1.0 / 3.0;
};

struct D3Q7 {
  static constexpr int Q = 7, DIM = 3;
  __device__ static constexpr int c(int i, int a) {
    constexpr int t[7][3] = {{0, 0, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    return t[i][a];
  }
  __device__ static constexpr double w(int i) { return i == 0 ? 0.25 : 0.125; }
  static constexpr double cs2 = 0.25;
};

template <class T>
struct AdeParams {
  int nx, ny, nz;
  int64_t n;
  T omega;
  T vu[3];
  const double* __restrict__ vf;  // [3][n] or nullptr (uniform vu)
  const uint8_t* __restrict__ mat;
  const uint8_t* __restrict__ lmask;
  const double* __restrict__ wall_C;
  unsigned periodic;
};

template <class T>
AdeParams<T> to_params(const AdeHost& h) {
  AdeParams<T> p;
  p.nx = h.nx;
  p.ny = h.ny;
  p.nz = h.nz;
  p.n = h.ncell;
  p.omega = (T)h.omega;
  for (int a = 0; a < 3; ++a) p.vu[a] = (T)h.vu[a];
  p.vf = h.vf;
  p.mat = h.mat;
  p.lmask = h.lmask;
  p.wall_C = h.wall_C;
  p.periodic = h.mat ? h.periodic : 7u;
  return p;
}

template <class L, class T>
__device__ __forceinline__ void equilibrium(T C, const T (&v)[3], T (&geq)[L::Q]) {
  constexpr T inv_cs2 = (T)(1.0 / L::cs2);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    T cv = T(0);
#pragma unroll
    for (int a = 0; a < L::DIM; ++a) {
      if (L::c(i, a) == 1) cv += v[a];
      if (L::c(i, a) == -1) cv -= v[a];
    }
    geq[i] = (T)L::w(i) * C * (T(1) + cv * inv_cs2);
  }
}

template <class T>
__device__ __forceinline__ void velocity(const AdeParams<T>& p, int64_t c, T (&v)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = p.vf ? (T)p.vf[a * p.n + c] : p.vu[a];
}

// BC = false: every cell bulk, every axis periodic (no mask, material or wall code).
template <class L, class T, bool BC>
__global__ void __launch_bounds__(256) k_ade_step(AdeParams<T> p, const T* __restrict__ src, T* __restrict__ dst) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.n) return;
  const int x = (int)(c % p.nx);
  const int64_t r = c / p.nx;
  const int y = (int)(r % p.ny);
  const int z = (int)(r / p.ny);
  T g[L::Q];
  T C = T(0);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    g[i] = src[i * p.n + c];
    C += g[i];
  }
  unsigned links = 0u;
  if (BC) {
    links = p.lmask[c];
    if (p.mat[c] != 1) {  // non-bulk cells keep their values
#pragma unroll
      for (int i = 0; i < L::Q; ++i) dst[i * p.n + c] = g[i];
      return;
    }
  }
  T v[3], geq[L::Q];
  velocity(p, c, v);
  equilibrium<L>(C, v, geq);
  const int xs[3] = {x == 0 ? p.nx - 1 : x - 1, x, x == p.nx - 1 ? 0 : x + 1};
  const int ys[3] = {y == 0 ? p.ny - 1 : y - 1, y, y == p.ny - 1 ? 0 : y + 1};
  const int zs[3] = {z == 0 ? p.nz - 1 : z - 1, z, z == p.nz - 1 ? 0 : z + 1};
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const T gs = g[i] - p.omega * (g[i] - geq[i]);
    const int64_t t = ((int64_t)zs[1 + L::c(i, 2)] * p.ny + ys[1 + L::c(i, 1)]) * p.nx + xs[1 + L::c(i, 0)];
    if (!BC || !(links & (1u << i))) {
      dst[i * p.n + t] = gs;
      continue;
    }
    // wall link: the target is a non-bulk cell, or outside the domain (the wrapped
    // index then names a cell on the far side, but the link leaves along a
    // non-periodic axis exactly when the unwrapped coordinate is out of range)
    const int q[3] = {x + L::c(i, 0), y + L::c(i, 1), z + L::c(i, 2)};
    const int e[3] = {p.nx, p.ny, p.nz};
    bool leaves = false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if ((q[a] < 0 || q[a] >= e[a]) && !(p.periodic & (1u << a))) leaves = true;
    const int m = leaves ? 0 : p.mat[t];
    const int o = i == 0 ? 0 : (i <= L::Q / 2 ? i + L::Q / 2 : i - L::Q / 2);
    if (m >= 2)
      dst[o * p.n + c] = -gs + T(2) * (T)L::w(i) * (T)p.wall_C[m];
    else
      dst[o * p.n + c] = gs;
  }
}

template <class L, class T>
__global__ void __launch_bounds__(256) k_ade_init(AdeParams<T> p, const double* __restrict__ Cin, T* __restrict__ g) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.n) return;
  T v[3], geq[L::Q];
  velocity(p, c, v);
  equilibrium<L>((T)Cin[c], v, geq);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) g[i * p.n + c] = geq[i];
}

template <class L, class T>
__global__ void __launch_bounds__(256) k_ade_density(AdeParams<T> p, const T* __restrict__ g, double* __restrict__ Cout) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.n) return;
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) s += (double)g[i * p.n + c];
  Cout[c] = s;
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

template <class L, class T>
cudaError_t step_t(const AdeHost& h, const void* src, void* dst) {
  if (h.mat)
    k_ade_step<L, T, true><<<blocks_for(h.ncell), 256, 0, h.stream>>>(to_params<T>(h), static_cast<const T*>(src),
                                                                        static_cast<T*>(dst));
  else
    k_ade_step<L, T, false><<<blocks_for(h.ncell), 256, 0, h.stream>>>(to_params<T>(h), static_cast<const T*>(src),
                                                                         static_cast<T*>(dst));
  return cudaGetLastError();
}

template <class L, class T>
cudaError_t init_t(const AdeHost& h, const double* C, void* g) {
  k_ade_init<L, T><<<blocks_for(h.ncell), 256, 0, h.stream>>>(to_params<T>(h), C, static_cast<T*>(g));
  return cudaGetLastError();
}

template <class L, class T>
cudaError_t density_t(const AdeHost& h, const void* g, double* C) {
  k_ade_density<L, T><<<blocks_for(h.ncell), 256, 0, h.stream>>>(to_params<T>(h), static_cast<const T*>(g), C);
  return cudaGetLastError();
}

}  // namespace

cudaError_t ade_step(const AdeHost& h, const void* src, void* dst) {
  if (h.q == 5) return h.f64 ? step_t<D2Q5, double>(h, src, dst) : step_t<D2Q5, float>(h, src, dst);
  return h.f64 ? step_t<D3Q7, double>(h, src, dst) : step_t<D3Q7, float>(h, src, dst);
}

cudaError_t ade_init(const AdeHost& h, const double* C, void* g) {
  if (h.q == 5) return h.f64 ? init_t<D2Q5, double>(h, C, g) : init_t<D2Q5, float>(h, C, g);
  return h.f64 ? init_t<D3Q7, double>(h, C, g) : init_t<D3Q7, float>(h, C, g);
}

cudaError_t ade_density(const AdeHost& h, const void* g, double* C) {
  if (h.q == 5) return h.f64 ? density_t<D2Q5, double>(h, g, C) : density_t<D2Q5, float>(h, g, C);
  return h.f64 ? density_t<D3Q7, double>(h, g, C) : density_t<D3Q7, float>(h, g, C);
}

}  // namespace olb
