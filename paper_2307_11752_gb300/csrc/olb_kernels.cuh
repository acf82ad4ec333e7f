// olb_kernels.cuh -- sm_103a kernels of the fused BGK collide-and-stream update.
//
// One thread updates one cell.  Populations are structure-of-arrays planes
// [q][cells] (x fastest) holding f_i - w_i ("weight-shifted": the rest state is
// all zero bits, and 16-bit storage spends its precision on the deviation from
// rest).  The update is bandwidth-bound (about 200 flops against 2 x q stored
// values per cell), so the design goal is one coalesced read and one coalesced
// write of every population per step and nothing else on the common path:
//   * bulk cells (all q neighbours fluid) take no branch on boundaries; periodic
//     axes are handled by wrapped row/column indices computed once per thread;
//   * cells next to a wall read one extra 32-bit mask with one bit per link;
//     moving-wall velocities are looked up only on those links;
//   * the streaming pattern is a template parameter: two-buffer pull (read the
//     neighbours, write the own cell) or the in-place AA pattern (even step: own
//     cell, swapped slots; odd step: read and write the neighbours' slots).
//
// The method (OpenLB user guide, arXiv 2307.11752):
//   collision  f*_i = f_i + omega (f^eq_i - f_i)           BGK equation and listing
//   forcing    + (1 - omega/2) w_i (3 (c_i - u') + 9 (c_i.u') c_i) . F,  u = (j + F/2)/rho   Eqs. FBD, dF
//   porosity   u' = gamma u in the equilibrium and forcing terms            section "Porous Media Model"
//   streaming  f_i(t+1, x + c_i) = f*_i(t, x)                               streaming equation
//   bounce-back (halfway) f_opp(i)(t+1, x) = f*_i(t, x) [- 6 w_i rho_x c_i.u_w on moving walls]
// with the second-order equilibrium
//   f^eq_i - w_i = w_i [(rho - 1) + rho (3 c_i.u' + 4.5 (c_i.u')^2 - 1.5 u'.u')].
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

#include "olb_internal.h"

// The generic (one cell per thread) BGK collision with omega w_k folded into the
// equilibrium's coefficients per weight class: fewer arithmetic instructions, which
// is what bounds the FP64 step on this GPU.
#ifndef OLB_FOLD_OMEGA_GENERIC
#define OLB_FOLD_OMEGA_GENERIC 1
#endif
// Resident blocks of 256 threads per SM that the step kernel is compiled for
// (bounds its registers: 65536 / (256 * blocks)).
#ifndef OLB_STEP_MIN_BLOCKS
#define OLB_STEP_MIN_BLOCKS 4
#endif
// FP64: 2 blocks (<= 128 registers, no spill; at 4 blocks it spills ~390 bytes per
// thread).  The FP64 step is bound by the FP64 pipe, which 16 warps per SM keep busy.
#ifndef OLB_STEP64_MIN_BLOCKS
#define OLB_STEP64_MIN_BLOCKS 2
#endif
// Same for the two-cells-per-thread step kernel (FP32 arithmetic), for FP32
// storage and for 16-bit storage (which needs more cells in flight per byte).
// FP32: 3 blocks (<= 80 registers) with the bounce-back stores first and their
// targets rebuilt from the coordinates (below).  Measured at 128^3 against 2
// blocks (128 registers, stores last): cavity pull 50.4 against 52.2 us, AA 55.3
// against 59.3 us (mean of the two half steps), TRT 50.8 against 53.2 us, the
// all-fluid box 47.5 against 48.6 us.
#ifndef OLB_PAIR_MIN_BLOCKS
#define OLB_PAIR_MIN_BLOCKS 3
#endif
// Use the boundary-capable instance of the paired kernel on every lattice (for
// measuring what the boundary code costs on lattices without walls).
#ifndef OLB_FORCE_WALLS
#define OLB_FORCE_WALLS 0
#endif
// 16-bit storage: 4 blocks (<= 64 registers).  Measured at 128^3: the all-fluid
// instance fits without spilling and runs 6% faster than at 3 blocks; the
// instance with walls spills 52 bytes and still runs 4% faster; 5 blocks (48
// registers) spills 160 bytes and runs 19% slower.
#ifndef OLB_PAIR16_MIN_BLOCKS
#define OLB_PAIR16_MIN_BLOCKS 4
#endif
#ifndef OLB_PAIR16_WALLS_MIN_BLOCKS
#define OLB_PAIR16_WALLS_MIN_BLOCKS 4
#endif
// The TRT instances at 3 blocks (<= 80 registers): at 4 they spill 212 bytes per
// thread; on the 128^3 cavity 37.8 against 44.2 us.
#ifndef OLB_PAIR16_TRT_MIN_BLOCKS
#define OLB_PAIR16_TRT_MIN_BLOCKS 3
#endif
// Order and addressing of the bounce-back stores of the paired kernel, per storage
// width: FIRST = before the own-slot stores (fewer live registers), COORDS = the
// target index rebuilt from the coordinates instead of kept from the loads.
#ifndef OLB_GHOST_FIRST16
#define OLB_GHOST_FIRST16 1
#endif
#ifndef OLB_GHOST_COORDS16
#define OLB_GHOST_COORDS16 1
#endif
#ifndef OLB_GHOST_FIRST32
#define OLB_GHOST_FIRST32 1
#endif
#ifndef OLB_GHOST_COORDS32
#define OLB_GHOST_COORDS32 1
#endif
// The pull step (two-buffer, state POST) of the paired kernel takes its populations
// through TMA tile copies into shared memory (olb_tma.cuh) where the lattice fits;
// tiles in flight per block for FP32 and for 16-bit storage.
#ifndef OLB_TMA
#define OLB_TMA 0
#endif
#ifndef OLB_TMA_STAGES32
#define OLB_TMA_STAGES32 2
#endif
#ifndef OLB_TMA_STAGES16
#define OLB_TMA_STAGES16 3
#endif
#ifndef OLB_TMA_WARP_ISSUE
#define OLB_TMA_WARP_ISSUE 1
#endif
// Launch the step kernels with programmatic dependent launch (each step's grid is
// scheduled while the previous one drains, and waits for it before touching memory).
#ifndef OLB_PDL
#define OLB_PDL 1
#endif

namespace olb {

// ---------------------------------------------------------------------------------
// Lattices.  D2Q9 as printed in the guide's "Descriptor" listing; D3Q19 with rest,
// then the nine velocities whose first non-zero component is -1, then their
// opposites (index i + 9 = -c_i).  Pairs (i, i + HALF) are opposite velocities.
// ---------------------------------------------------------------------------------
struct D2Q9 {
  static constexpr int Q = 9, DIM = 2, HALF = 4;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0},  {-1, 1, 0}, {-1, 0, 0}, {-1, -1, 0}, {0, -1, 0},
                             {1, -1, 0}, {1, 0, 0},  {1, 1, 0},  {0, 1, 0}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : ((i % 2) == 0 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

struct D3Q19 {
  static constexpr int Q = 19, DIM = 3, HALF = 9;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[19][3] = {{0, 0, 0},   {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {-1, -1, 0},
                              {-1, 1, 0},  {-1, 0, -1}, {-1, 0, 1}, {0, -1, -1}, {0, -1, 1},
                              {1, 0, 0},   {0, 1, 0},  {0, 0, 1},  {1, 1, 0},  {1, -1, 0},
                              {1, 0, 1},   {1, 0, -1}, {0, 1, 1},  {0, 1, -1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (((i - 1) % 9) < 3 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

template <class L>
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= L::HALF ? i + L::HALF : i - L::HALF);
}

// Link word of a cell, read by the step kernel together with the populations.
//   fluid cell:  kWordFluid | [kWordMoving] | bit i for every link whose target
//                x + c_i is a non-fluid cell of the lattice (bounce-back link)
//   other cell:  bit i when x + c_i is a fluid cell
constexpr uint32_t kWordFluid = 1u << 31;
constexpr uint32_t kWordMoving = 1u << 30;  // a bounce-back link hits a moving wall
constexpr uint32_t kWordLinks = (1u << 19) - 1;
// Moving links of a fluid cell in plane form (bits 19..29): when the moving links
// are exactly the wall links with c_i[a] == s and all hit one material m, bits
// 19..21 hold 1 + 2a + (s > 0) and bits 22..29 hold m; the step kernel then takes
// the wall term from the cell's own word instead of loading each neighbour's
// material.  Plane code 0: load the materials (any other arrangement).
constexpr int kWordPlaneShift = 19;
constexpr int kWordMatShift = 22;

// Non-fluid cells also store zeros into the slots that no fluid neighbour fills,
// so that every memory sector of a step's output is written in full.
#ifndef OLB_SOLID_FILL
#define OLB_SOLID_FILL 0
#endif

// Programmatic dependent launch.  A step grid launched with the programmatic
// stream-serialization attribute can be scheduled before the previous step's grid
// has finished.  griddepcontrol.wait blocks until every prerequisite grid has
// completed and its memory operations are visible (it returns at once when the
// grid was launched without the attribute), so it comes before the first global
// access; launch_dependents then allows the next step's grid to be scheduled
// into the SM slots this grid's blocks free as they retire.
__device__ __forceinline__ void pdl_wait() {
#if OLB_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_release() {
#if OLB_PDL
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_wait_then_release() {
  pdl_wait();
  pdl_release();
}

// Launch `kernel` on `stream` with `smem` bytes of dynamic shared memory, with the
// programmatic stream-serialization attribute when OLB_PDL is on.
template <class... Exp, class... Act>
cudaError_t launch_step(void (*kernel)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                        Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = tma_setting("OLB_PDL", OLB_PDL) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Act>(args)...);
}

// ---------------------------------------------------------------------------------
// Storage types: load/store with conversion to the compute type.
// ---------------------------------------------------------------------------------
template <class S>
struct Store;
template <>
struct Store<double> {
  using C = double;
  __device__ static C ld(const double* p) { return *p; }
  __device__ static void st(double* p, C v) { *p = v; }
};
template <>
struct Store<float> {
  using C = float;
  __device__ static C ld(const float* p) { return *p; }
  __device__ static void st(float* p, C v) { *p = v; }
};
// FP16 holds (f - w) * 2^12: an exact power-of-two scale that moves deviations
// down to ~1e-8 out of FP16's subnormal range (normal range starts at 6.1e-5);
// deviations up to 16 stay finite, far beyond any stable state.
template <>
struct Store<__half> {
  using C = float;
  static constexpr float kScale = 4096.0f, kInvScale = 1.0f / 4096.0f;
  __device__ static C ld(const __half* p) { return __half2float(*p) * kInvScale; }
  __device__ static void st(__half* p, C v) { *p = __float2half_rn(v * kScale); }
};
template <>
struct Store<__nv_bfloat16> {
  using C = float;
  __device__ static C ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ static void st(__nv_bfloat16* p, C v) { *p = __float2bfloat16_rn(v); }
};

// Kernel parameters in the compute type C.
template <class C>
struct Params {
  int nx, ny, nz, ncell;
  int pitch;  // elements between population planes (>= ncell; canonical arrays use ncell)
  unsigned periodic;
  int all_fluid;  // every cell fluid and every axis periodic: no class reads
  const uint8_t* __restrict__ cls;
  const uint32_t* __restrict__ wmask;  // per cell: bit i set when x - c_i is not a fluid cell
  const uint8_t* __restrict__ mat;
  const double* __restrict__ wall_u;  // [256][4]
  int moving;
  C omega, half_force[3], force[3];
  C omega_minus;  // TRT: relaxation rate of the odd part (omega is the even rate)
  C domega_minus;  // TRT: d omega_minus / d omega at fixed magic parameter (BGK: 1)
  int forced;  // a uniform force or a force field is set
  // per-cell force density [3][ncell] in the compute type, or null (the uniform force)
  const C* __restrict__ ffield;
  const C* __restrict__ gamma;
  // per cell: bit i set when x + c_i is a non-fluid cell of the lattice (a wall
  // link whose bounced population is stored in that cell)
  const uint32_t* __restrict__ pmask;
  // per cell link word of the step kernel (see kWordFluid)
  const uint32_t* __restrict__ word;
  int outside_links;  // some fluid cell has a link leaving the domain
  // step-kernel grid: gx * gy * nz tiles of (1 << tile_shift) x (256 >> tile_shift)
  int gx, gy, tile_shift;
  int y0, z0, y1, z1;  // rows covered by the step grid
  int az0, az1;        // active planes: statistics count cells with z in [az0, az1]
  const float* __restrict__ wall_f;  // [256][20]: 6 w_i (c_i . u_w) rounded once to FP32
};

template <class C>
Params<C> to_params(const HostParams& h) {
  Params<C> p;
  p.nx = h.nx;
  p.ny = h.ny;
  p.nz = h.nz;
  p.ncell = h.ncell;
  p.pitch = h.pitch;
  p.periodic = h.periodic;
  p.all_fluid = 0;
  p.cls = h.cls;
  p.wmask = h.wmask;
  p.mat = h.mat;
  p.wall_u = h.wall_u;
  p.wall_f = h.wall_f;
  p.moving = h.moving;
  p.omega = (C)h.omega;
  p.omega_minus = (C)h.omega_minus;
  p.domega_minus = (C)h.domega_minus;
  for (int a = 0; a < 3; ++a) {
    p.force[a] = (C)h.force[a];
    p.half_force[a] = (C)(0.5 * h.force[a]);
  }
  p.forced = h.forced || h.ffield != nullptr;
  p.ffield = reinterpret_cast<const C*>(h.ffield);
  p.gamma = reinterpret_cast<const C*>(h.gamma);
  p.pmask = h.pmask;
  p.word = h.word;
  p.outside_links = h.outside_links;
  p.y0 = h.y0;
  p.y1 = h.y1;
  p.z0 = h.z0;
  p.z1 = h.z1;
  p.az0 = h.az0;
  p.az1 = h.az1;
  const StepGrid sg = make_step_grid(h, false);
  p.gx = sg.gx;
  p.gy = sg.gy;
  p.tile_shift = sg.tile_shift;
  return p;
}

// ---------------------------------------------------------------------------------
// Neighbourhood of one cell: wrapped x indices and row bases for the 3 x 3
// (dy, dz) offsets; at(dx, dy, dz) is the flat index of cell + (dx, dy, dz).
// ---------------------------------------------------------------------------------
struct Nbr {
  int x, y, z, cell;
  int xo[3];
  int row[3][3];
  __device__ __forceinline__ int at(int dx, int dy, int dz) const {
    return row[dz + 1][dy + 1] + xo[dx + 1];
  }
};

template <class L, class C>
__device__ __forceinline__ Nbr make_nbr(const Params<C>& p, int x, int y, int z) {
  Nbr n;
  n.x = x;
  n.y = y;
  n.z = z;
  n.xo[0] = x == 0 ? p.nx - 1 : x - 1;
  n.xo[1] = x;
  n.xo[2] = x == p.nx - 1 ? 0 : x + 1;
  const int ys[3] = {y == 0 ? p.ny - 1 : y - 1, y, y == p.ny - 1 ? 0 : y + 1};
  int zs[3] = {z, z, z};
  if (L::DIM == 3) {
    zs[0] = z == 0 ? p.nz - 1 : z - 1;
    zs[2] = z == p.nz - 1 ? 0 : z + 1;
  }
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) n.row[dz][dy] = (zs[dz] * p.ny + ys[dy]) * p.nx;
  n.cell = n.row[1][1] + x;
  return n;
}

// Material number of the cell at offset (dx, dy, dz); 0 (void) outside the
// domain along a non-periodic axis.  Only used on moving-wall links.
template <class C>
__device__ __forceinline__ int link_material(const Params<C>& p, const Nbr& n, int dx, int dy,
                                             int dz) {
  int q[3] = {n.x + dx, n.y + dy, n.z + dz};
  const int e[3] = {p.nx, p.ny, p.nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (q[a] < 0 || q[a] >= e[a]) {
      if (!(p.periodic & (1u << a))) return 0;
      q[a] = q[a] < 0 ? q[a] + e[a] : q[a] - e[a];
    }
  }
  return p.mat[(q[2] * p.ny + q[1]) * p.nx + q[0]];
}

// 6 w_i (c_i . u_w) of wall material m.  The FP32 paths read it from the table
// the host fills when a wall velocity is set (the same double expression, rounded
// once), so that no FP64 instruction runs in them: FP64 issues at a small fraction
// of the FP32 rate on sm_103a, and the cells next to a moving wall sit together in
// the last blocks of the grid, where that work would lengthen the kernel's tail.
template <class L, class C>
__device__ __forceinline__ C wall_term(const Params<C>& p, int i, int m) {
  if constexpr (sizeof(C) == sizeof(float)) {
    return p.wall_f[20 * m + i];
  } else {
    const double* u = p.wall_u + 4 * m;
    double cu = L::c(i, 0) * u[0] + L::c(i, 1) * u[1] + L::c(i, 2) * u[2];
    return (C)(6.0 * L::w(i) * cu);
  }
}

// Force density of a cell: the per-cell field when one is set, else the uniform force.
template <class C>
__device__ __forceinline__ void force_at(const Params<C>& p, int cell, C (&F)[3]) {
  if (p.ffield) {
    const size_t N = (size_t)p.ncell;
    F[0] = p.ffield[cell];
    F[1] = p.ffield[N + cell];
    F[2] = p.ffield[2 * N + cell];
  } else {
    F[0] = p.force[0];
    F[1] = p.force[1];
    F[2] = p.force[2];
  }
}

// ---------------------------------------------------------------------------------
// Gather f(t) of one cell (shifted values, compute type) from a buffer in
// representation G:
//   G_OWN        f_i(x) = slot i of x                         (state PRE)
//   G_PULL       f_i(x) = slot i of x - c_i                   (state POST)
//   G_PULL_SWAP  f_i(x) = slot opp(i) of x - c_i              (state AA_ODD)
// Bounce-back needs no special case here: when x - c_i is a wall cell, the step
// that wrote the buffer stored the bounced population (moving-wall term
// included) in that wall cell's slot, which only x writes and only x reads (see
// scatter).  Only links that leave the domain along a non-periodic axis have no
// cell to hold it; cells with such links (class 3) take them from their own
// slots in gather_outside.  Every index is wrapped, so the bulk loads are valid
// for every cell and never wait for the cell class.
// ---------------------------------------------------------------------------------
template <class L, class S, int G>
__device__ __forceinline__ void gather_bulk(const Params<typename Store<S>::C>& p, const S* src,
                                            const Nbr& n, typename Store<S>::C (&f)[L::Q]) {
  const size_t N = (size_t)p.pitch;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    if constexpr (G == G_OWN) {
      f[i] = Store<S>::ld(src + i * N + n.cell);
    } else {
      const int slot = (G == G_PULL) ? i : opp<L>(i);
      f[i] = Store<S>::ld(src + slot * N + n.at(-L::c(i, 0), -L::c(i, 1), -L::c(i, 2)));
    }
  }
}

// True when cell + (dx, dy, dz) leaves the domain along a non-periodic axis.
template <class C>
__device__ __forceinline__ bool outside(const Params<C>& p, const Nbr& n, int dx, int dy, int dz) {
  const int q[3] = {n.x + dx, n.y + dy, n.z + dz};
  const int e[3] = {p.nx, p.ny, p.nz};
  bool out = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (!(p.periodic & (1u << a)) && (q[a] < 0 || q[a] >= e[a])) out = true;
  return out;
}

template <class L, class S, int G>
__device__ __forceinline__ void gather_outside(const Params<typename Store<S>::C>& p, const S* src,
                                               const Nbr& n, typename Store<S>::C (&f)[L::Q]) {
  if constexpr (G != G_OWN) {
    const size_t N = (size_t)p.pitch;
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
      if (outside(p, n, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2))) {
        // no-slip bounce-back at the domain edge: the population that left x
        // towards the edge, from x's own slots
        const int own = (G == G_PULL) ? opp<L>(i) : i;
        f[i] = Store<S>::ld(src + own * N + n.cell);
      }
    }
  }
}

template <class L, class S, int G>
__device__ __forceinline__ void gather(const Params<typename Store<S>::C>& p, const S* src,
                                       const Nbr& n, int cls,
                                       typename Store<S>::C (&f)[L::Q]) {
  gather_bulk<L, S, G>(p, src, n, f);
  if (cls == 3) gather_outside<L, S, G>(p, src, n, f);
}

// ---------------------------------------------------------------------------------
// Moments and collision on shifted populations.
// ---------------------------------------------------------------------------------
template <class L, class C>
__device__ __forceinline__ void moments(const C (&f)[L::Q], C& drho, C (&j)[3]) {
  drho = f[0];
  j[0] = j[1] = j[2] = C(0);
#pragma unroll
  for (int k = 1; k <= L::HALF; ++k) {
    const int kp = k + L::HALF;  // c_kp = -c_k
    const C s = f[k] + f[kp];
    const C a = f[kp] - f[k];
    drho += s;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (L::c(kp, d) == 1) j[d] += a;
      if (L::c(kp, d) == -1) j[d] -= a;
    }
  }
}

// BGK collision (+ Guo forcing, + porosity) in place.  Returns rho and the
// unscaled velocity u = (j + F/2)/rho through the out parameters.
// TRT = true: the two-relaxation-time operator (collision::TRT of the dynamics
// tuples, section "Dynamics"): for each pair (i, opp(i)) the even part
// f+ = (f_i + f_opp(i))/2 relaxes to the even part of f^eq at omega, the odd part
// f- at omega_minus, and the Guo source is split the same way with factors
// (1 - omega/2) and (1 - omega_minus/2).
template <class L, class C, bool TRT = false>
__device__ __forceinline__ void collide(const Params<C>& p, C gamma, const C (&F)[3], C (&f)[L::Q], C drho,
                                        const C (&j)[3], C& rho_out, C (&u_out)[3]) {
  const C rho = C(1) + drho;
  const C inv = C(1) / rho;
  C u[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) u[d] = (j[d] + C(0.5) * F[d]) * inv;
  rho_out = rho;
  u_out[0] = u[0];
  u_out[1] = u[1];
  u_out[2] = u[2];
  const C up[3] = {gamma * u[0], gamma * u[1], gamma * u[2]};
  const C usq = up[0] * up[0] + up[1] * up[1] + (L::DIM == 3 ? up[2] * up[2] : C(0));
  const C om = p.omega;
  const C rs = C(1.5) * rho * usq;
  const C gf = C(1) - C(0.5) * om;
  C uF = C(0);
  if (p.forced) uF = up[0] * F[0] + up[1] * F[1] + up[2] * F[2];
  {
    const C w0 = (C)L::w(0);
    C feq = w0 * (drho - rs);
    f[0] += om * (feq - f[0]);
    if (p.forced) f[0] -= gf * w0 * C(3) * uF;
  }
#pragma unroll
  for (int k = 1; k <= L::HALF; ++k) {
    const int kp = k + L::HALF;
    const C wk = (C)L::w(k);
    C cu = C(0), cF = C(0);
#pragma unroll
    for (int d = 0; d < L::DIM; ++d) {
      if (L::c(kp, d) == 1) {
        cu += up[d];
        cF += F[d];
      }
      if (L::c(kp, d) == -1) {
        cu -= up[d];
        cF -= F[d];
      }
    }
    if (!TRT && OLB_FOLD_OMEGA_GENERIC) {
      // omega (feq_k - f_k) with omega w_k folded into the equilibrium's coefficients
      // (the products are common to the directions of equal weight):
      //   Aw = omega w_k (drho - 1.5 rho u'^2), Bw = 4.5 omega w_k rho, Tw = 3 omega w_k rho
      const C omw = om * wk;
      const C symw = omw * (drho - rs) + (omw * C(4.5)) * rho * (cu * cu);
      const C antiw = (omw * C(3)) * rho * cu;
      f[kp] = (C(1) - om) * f[kp] + (symw + antiw);
      f[k] = (C(1) - om) * f[k] + (symw - antiw);
      if (p.forced) {
        const C gs = gf * wk * (C(9) * cu * cF - C(3) * uF);
        const C ga = gf * wk * C(3) * cF;
        f[kp] += gs + ga;
        f[k] += gs - ga;
      }
      continue;
    }
    const C sym = wk * (drho + rho * (C(4.5) * cu * cu) - rs);
    const C anti = wk * C(3) * rho * cu;
    if (TRT) {
      const C om_m = p.omega_minus;
      const C even = om * (C(0.5) * (f[kp] + f[k]) - sym);
      const C odd = om_m * (C(0.5) * (f[kp] - f[k]) - anti);
      f[kp] -= even + odd;
      f[k] -= even - odd;
      if (p.forced) {
        const C gs = gf * wk * (C(9) * cu * cF - C(3) * uF);
        const C ga = (C(1) - C(0.5) * om_m) * wk * C(3) * cF;
        f[kp] += gs + ga;
        f[k] += gs - ga;
      }
      continue;
    }
    f[kp] += om * (sym + anti - f[kp]);
    f[k] += om * (sym - anti - f[k]);
    if (p.forced) {
      const C gs = gf * wk * (C(9) * cu * cF - C(3) * uF);
      const C ga = gf * wk * C(3) * cF;
      f[kp] += gs + ga;
      f[k] += gs - ga;
    }
  }
}

// ---------------------------------------------------------------------------------
// Scatter post-collision values f*_i(x) to a buffer with pattern SC.
//   S_OWN       slot i of x                         -> state POST (next gather G_PULL)
//   S_OWN_SWAP  slot opp(i) of x                    -> state AA_ODD (next gather G_PULL_SWAP)
//   S_PUSH      slot i of x + c_i                   -> state PRE (next gather G_OWN)
// Halfway bounce-back (class >= 2, `pm` = links whose target x + c_i is a wall
// cell of the lattice): the bounced population f*_i(x) - 6 w_i rho_x c_i.u_w is
// what x will read for direction opp(i) at the next step.  S_OWN and S_OWN_SWAP
// store it in the wall cell x + c_i, in the slot the next gather of x reads
// there (opp(i) for G_PULL, i for G_PULL_SWAP); S_PUSH stores it in x's own
// slot opp(i).  Links leaving the domain (class 3) bounce through x's own slots.
// ---------------------------------------------------------------------------------
template <class L, class S, int SC>
__device__ __forceinline__ void scatter(const Params<typename Store<S>::C>& p, S* dst,
                                        const Nbr& n, int cls, uint32_t pm,
                                        const typename Store<S>::C (&f)[L::Q],
                                        typename Store<S>::C rho) {
  using C = typename Store<S>::C;
  const size_t N = (size_t)p.pitch;
  if (SC == S_OWN || SC == S_OWN_SWAP) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int slot = (SC == S_OWN) ? i : opp<L>(i);
      Store<S>::st(dst + slot * N + n.cell, f[i]);
    }
    if (cls >= 2) {
#pragma unroll
      for (int i = 1; i < L::Q; ++i) {
        if (pm & (1u << i)) {
          C v = f[i];
          if (pm & kWordMoving) {
            const int wm = p.mat[n.at(L::c(i, 0), L::c(i, 1), L::c(i, 2))];
            if (wm >= 3) v -= rho * wall_term<L>(p, i, wm);
          }
          const int slot = (SC == S_OWN) ? opp<L>(i) : i;
          Store<S>::st(dst + slot * N + n.at(L::c(i, 0), L::c(i, 1), L::c(i, 2)), v);
        }
      }
    }
  } else {  // S_PUSH
    if (cls == 1) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i)
        Store<S>::st(dst + i * N + n.at(L::c(i, 0), L::c(i, 1), L::c(i, 2)), f[i]);
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const bool wall = i != 0 && (pm & (1u << i));
        const bool edge = i != 0 && cls == 3 && outside(p, n, L::c(i, 0), L::c(i, 1), L::c(i, 2));
        // (pm carries only link bits 0..18 and kWordMoving)
        if (wall || edge) {
          C v = f[i];
          if (wall && (pm & kWordMoving)) {
            const int wm = p.mat[n.at(L::c(i, 0), L::c(i, 1), L::c(i, 2))];
            if (wm >= 3) v -= rho * wall_term<L>(p, i, wm);
          }
          Store<S>::st(dst + opp<L>(i) * N + n.cell, v);
        } else {
          Store<S>::st(dst + i * N + n.at(L::c(i, 0), L::c(i, 1), L::c(i, 2)), f[i]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Block reduction of 8 per-thread values into one row of `partials`:
// entries 0..4 and 6..7 are sums, entry 5 is a maximum.  Warp stage in the compute
// type, block and global stages in double.
// ---------------------------------------------------------------------------------
template <class C>
__device__ __forceinline__ void block_reduce_row(C (&v)[8], double* row, bool accumulate) {
  __shared__ double sh[32][8];
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      C other = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = (k == 5) ? (other > v[k] ? other : v[k]) : v[k] + other;
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) sh[warp][k] = (double)v[k];
  }
  __syncthreads();
  if (tid < 8) {
    double acc = sh[0][tid];
    for (int w = 1; w < nwarps; ++w) acc = (tid == 5) ? fmax(acc, sh[w][tid]) : acc + sh[w][tid];
    if (accumulate) {
      row[tid] = (tid == 5) ? fmax(row[tid], acc) : row[tid] + acc;
    } else {
      row[tid] = acc;
    }
  }
}

__device__ __forceinline__ int64_t block_linear() {
  return (int64_t)blockIdx.x + (int64_t)gridDim.x * ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
}

// Per-cell statistics contribution: {rho - 1, j_x, j_y, j_z, |u|^2/2, |u|, bad, 1}.
template <class C>
__device__ __forceinline__ void stats_of(C drho, const C (&j)[3], const C (&u)[3], C (&v)[8]) {
  if (isfinite(drho) && isfinite(j[0]) && isfinite(j[1]) && isfinite(j[2])) {
    const C uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    v[0] = drho;
    v[1] = j[0];
    v[2] = j[1];
    v[3] = j[2];
    v[4] = C(0.5) * uu;
    v[5] = sqrt(uu);
    v[6] = C(0);
    v[7] = C(1);
  } else {
    v[0] = v[1] = v[2] = v[3] = v[4] = v[5] = C(0);
    v[6] = C(1);
    v[7] = C(0);
  }
}

// ---------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------
// Zero the slots of a non-fluid cell that no fluid neighbour writes in this step
// (its bounce-back slots are written by the neighbours).  `nb` = bit k when
// x + c_k is fluid.  Pull (S_OWN): slot k is filled by x + c_k.  AA (S_OWN_SWAP,
// S_PUSH): slot k is filled by, or read in this step by, x - c_k.
template <class L, class S, int SC>
__device__ __forceinline__ void solid_fill(const Params<typename Store<S>::C>& p, S* dst,
                                           const Nbr& n, uint32_t nb) {
  const size_t N = (size_t)p.pitch;
#pragma unroll
  for (int k = 0; k < L::Q; ++k) {
    const int b = (SC == S_OWN) ? k : opp<L>(k);
    if (k == 0 || !(nb & (1u << b))) Store<S>::st(dst + k * N + n.cell, typename Store<S>::C(0));
  }
}

// True when the cell lies on a face of the domain along a non-periodic axis.
template <class L, class C>
__device__ __forceinline__ bool on_edge(const Params<C>& p, int x, int y, int z) {
  return (!(p.periodic & 1u) && (x == 0 || x == p.nx - 1)) ||
         (!(p.periodic & 2u) && (y == 0 || y == p.ny - 1)) ||
         (L::DIM == 3 && !(p.periodic & 4u) && (z == 0 || z == p.nz - 1));
}

// One collide-and-stream step.  Blocks tile the lattice in rows of up to 256
// cells along x.  Each thread loads its cell's link word together with the
// populations -- no load depends on another -- so a single memory latency covers
// the cell; it collides and stores.  Links leaving the domain (only when some
// fluid cell touches a non-periodic domain face) are recognised from the
// coordinates, again without waiting for a load.
template <class L, class S, int G, int SC, bool STATS, bool TRT>
__global__ void __launch_bounds__(256, std::is_same<S, double>::value ? OLB_STEP64_MIN_BLOCKS : OLB_STEP_MIN_BLOCKS)
    k_step(Params<typename Store<S>::C> p, const S* src, S* dst, double* partials) {
  using C = typename Store<S>::C;
  C sv[8] = {C(0), C(0), C(0), C(0), C(0), C(0), C(0), C(0)};
  const int tid = threadIdx.x;
  pdl_wait_then_release();
  const int z = p.z0 + blockIdx.z;
  const int x = (blockIdx.x << p.tile_shift) + (tid & ((1 << p.tile_shift) - 1));
  const int y = p.y0 + blockIdx.y * (256 >> p.tile_shift) + (tid >> p.tile_shift);
  if (x < p.nx && y <= p.y1) {
    const Nbr n = make_nbr<L>(p, x, y, z);
    const uint32_t w = p.all_fluid ? kWordFluid : p.word[n.cell];
    C f[L::Q];
    gather_bulk<L, S, G>(p, src, n, f);
    const C gamma = p.gamma ? p.gamma[n.cell] : C(1);
    C F[3];
    force_at(p, n.cell, F);
    const bool edge = p.outside_links && on_edge<L>(p, x, y, z);
    if (edge) gather_outside<L, S, G>(p, src, n, f);
    C drho, j[3], rho, u[3];
    moments<L>(f, drho, j);
    collide<L, C, TRT>(p, gamma, F, f, drho, j, rho, u);
    if (w & kWordFluid) {
      const uint32_t pm = w & (kWordLinks | kWordMoving);
      const int cls = edge ? 3 : (pm ? 2 : 1);
      scatter<L, S, SC>(p, dst, n, cls, pm, f, rho);
      if (STATS) stats_of(drho, j, u, sv);
    } else if (OLB_SOLID_FILL) {
      solid_fill<L, S, SC>(p, dst, n, w & kWordLinks);
    }
  }
  if (STATS) block_reduce_row(sv, partials + 8 * block_linear(), false);
}

// Canonical f(t) = f_shifted + w in double ([q][cells]); non-fluid cells 0.
template <class L, class S, int G>
__global__ void __launch_bounds__(256) k_to_f64(Params<typename Store<S>::C> p, const S* src, double* out) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const Nbr n = make_nbr<L>(p, x, y, blockIdx.z);
  const int cls = p.all_fluid ? 1 : p.cls[n.cell];
  const size_t N = (size_t)p.ncell;
  if (cls == 0) {
#pragma unroll
    for (int i = 0; i < L::Q; ++i) out[i * N + n.cell] = 0.0;
    return;
  }
  C f[L::Q];
  gather<L, S, G>(p, src, n, cls, f);
#pragma unroll
  for (int i = 0; i < L::Q; ++i) out[i * N + n.cell] = (double)f[i] + L::w(i);
}

template <class L, class S, int G>
__global__ void __launch_bounds__(256) k_moments(Params<typename Store<S>::C> p, const S* src, double* rho_out,
                                                 double* u_out) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const Nbr n = make_nbr<L>(p, x, y, blockIdx.z);
  const int cls = p.all_fluid ? 1 : p.cls[n.cell];
  const size_t N = (size_t)p.ncell;
  double r = 0.0, u[3] = {0.0, 0.0, 0.0};
  if (cls != 0) {
    C f[L::Q];
    gather<L, S, G>(p, src, n, cls, f);
    C drho, j[3], F[3];
    moments<L>(f, drho, j);
    force_at(p, n.cell, F);
    const C rho = C(1) + drho;
    r = (double)rho;
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = (double)((j[d] + C(0.5) * F[d]) / rho);
  }
  if (rho_out) rho_out[n.cell] = r;
  if (u_out) {
#pragma unroll
    for (int d = 0; d < 3; ++d) u_out[d * N + n.cell] = u[d];
  }
}

template <class L, class S, int G>
__global__ void __launch_bounds__(256) k_stats(Params<typename Store<S>::C> p, const S* src, double* partials) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  C sv[8] = {C(0), C(0), C(0), C(0), C(0), C(0), C(0), C(0)};
  if (x < p.nx && y < p.ny && (int)blockIdx.z >= p.az0 && (int)blockIdx.z <= p.az1) {
    const Nbr n = make_nbr<L>(p, x, y, blockIdx.z);
    const int cls = p.all_fluid ? 1 : p.cls[n.cell];
    if (cls != 0) {
      C f[L::Q];
      gather<L, S, G>(p, src, n, cls, f);
      C drho, j[3], F[3];
      moments<L>(f, drho, j);
      force_at(p, n.cell, F);
      const C rho = C(1) + drho;
      C u[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) u[d] = (j[d] + C(0.5) * F[d]) / rho;
      stats_of(drho, j, u, sv);
    }
  }
  block_reduce_row(sv, partials + 8 * block_linear(), false);
}

// Stored (shifted) populations from canonical double populations, own slots.
template <class L, class S>
__global__ void __launch_bounds__(256) k_from_f64(Params<typename Store<S>::C> p, const double* f, S* dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int cell = (blockIdx.z * p.ny + y) * p.nx + x;
  const size_t N = (size_t)p.ncell;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) Store<S>::st(dst + i * (size_t)p.pitch + cell, (typename Store<S>::C)(f[i * N + cell] - L::w(i)));
}

// Equilibrium initialisation f = f^eq(rho, u) (rho, u nullable: 1, 0).
template <class L, class S>
__global__ void __launch_bounds__(256) k_init_eq(Params<typename Store<S>::C> p, const double* rho_in,
                                                 const double* u_in, S* dst) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int cell = (blockIdx.z * p.ny + y) * p.nx + x;
  const size_t N = (size_t)p.ncell;
  const C rho = rho_in ? (C)rho_in[cell] : C(1);
  const C drho = rho_in ? (C)(rho_in[cell] - 1.0) : C(0);
  C u[3] = {C(0), C(0), C(0)};
  if (u_in) {
#pragma unroll
    for (int d = 0; d < L::DIM; ++d) u[d] = (C)u_in[d * N + cell];
  }
  const C usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    const C cu = L::c(i, 0) * u[0] + L::c(i, 1) * u[1] + L::c(i, 2) * u[2];
    const C feq = (C)L::w(i) * (drho + rho * (C(3) * cu + C(4.5) * cu * cu - C(1.5) * usq));
    Store<S>::st(dst + i * (size_t)p.pitch + cell, feq);
  }
}

template <class L, class S>
__global__ void __launch_bounds__(256) k_perturb(Params<typename Store<S>::C> p, const double* df, S* dst) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int cell = (blockIdx.z * p.ny + y) * p.nx + x;
  if (!p.all_fluid && p.cls[cell] == 0) return;
  const size_t N = (size_t)p.ncell;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    S* q = dst + i * (size_t)p.pitch + cell;
    Store<S>::st(q, (C)((double)Store<S>::ld(q) + df[i * N + cell]));
  }
}

// Rewrite a state in representation G as PRE (own slots) into another buffer.
template <class L, class S, int G>
__global__ void __launch_bounds__(256) k_materialize(Params<typename Store<S>::C> p, const S* src, S* dst) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const Nbr n = make_nbr<L>(p, x, y, blockIdx.z);
  const int cls = p.all_fluid ? 1 : p.cls[n.cell];
  if (cls == 0) return;
  C f[L::Q];
  gather<L, S, G>(p, src, n, cls, f);
  const size_t N = (size_t)p.pitch;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) Store<S>::st(dst + i * N + n.cell, f[i]);
}

// ---------------------------------------------------------------------------------
// Adjoint.  One reverse step maps lam^{n+1} (adjoint of the pre-collision state
// f(n+1), own slots) to lam^n, given f(n):
//   lam*_i(x) = lam^{n+1}_i(x + c_i)  (fluid neighbour)  |  lam^{n+1}_opp(i)(x)  (wall link)
//   lam^n_i   = (1 - omega) lam*_i + omega A + (gamma/rho) B.(c_i - u) + D
// with mu_k = w_k lam*_k and its moments m0 = sum mu, m1 = sum mu c, m2 = sum mu c c:
//   A = m0 (1 - 1.5 u'.u') + 3 m1.u' + 4.5 u'.m2.u'                (= sum lam*_k f^eq_k / rho)
//   B = omega rho (3 m1 + 9 m2 u' - 3 m0 u') + (1 - omega/2)(9 m2 F - 3 m0 F)
//   D = sum over moving-wall links of lam*_i (-6 w_i c_i.u_w)      (density in the wall term)
// and the gradient contributions
//   dL/dgamma(x) += B.u,
//   dL/domega    += -sum lam*_k f_k + rho A - (3 m1.F - 3 m0 u'.F + 9 u'.m2.F)/2,
//   dL/dF(x)     += (gamma/(2 rho)) B + (1 - omega/2)(3 m1 - 3 m0 u' + 9 m2 u')
// (F(x) the cell's force density: through u = (j + F/2)/rho, and explicitly in the
// Guo source).
// TRT = true (the two-relaxation-time collision): the relaxation and the source act
// on the even and odd parts of each pair (i, opp(i)) with omega+ = omega,
// omega- = omega_minus and (1 - omega+-/2).  The even part of lam* carries m0 and
// m2, the odd part m1, so the adjoint is the one above with omega on m1 replaced by
// omega- (in A and B; the source's derivative holds no m1), the own-population term
// lam*_i - omega+ lam*+_i - omega- lam*-_i, and, for dL/domega at fixed magic
// parameter, m1 and the odd part of sum lam* f scaled by d omega- / d omega.
// ---------------------------------------------------------------------------------
template <class S>
struct LambdaOf {
  using T = float;
};
template <>
struct LambdaOf<double> {
  using T = double;
};

template <class L, class S, int G, bool TRT>
__global__ void __launch_bounds__(256) k_adjoint(Params<typename Store<S>::C> p, const S* state,
                                                 const typename LambdaOf<S>::T* __restrict__ lam_in,
                                                 typename LambdaOf<S>::T* __restrict__ lam_out,
                                                 double* dgamma, double* dforce, double* partials) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const size_t N = (size_t)p.pitch;
  C sv[8] = {C(0), C(0), C(0), C(0), C(0), C(0), C(0), C(0)};
  pdl_wait_then_release();  // launched like the step kernels (the sweep alternates them)
  if (x < p.nx && y < p.ny) {
    const Nbr n = make_nbr<L>(p, x, y, blockIdx.z);
    const int cls = p.all_fluid ? 1 : p.cls[n.cell];
    if (cls != 0) {
      // lam* = S^T lam^{n+1}
      C ls[L::Q];
      C direct = C(0);
      if (cls == 1) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
          ls[i] = (C)lam_in[i * N + n.at(L::c(i, 0), L::c(i, 1), L::c(i, 2))];
      } else {
        const uint32_t m = p.wmask[n.cell];
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
          if (i != 0 && (m & (1u << opp<L>(i)))) {
            ls[i] = (C)lam_in[opp<L>(i) * N + n.cell];
            if (p.moving) {
              const int wm = link_material(p, n, L::c(i, 0), L::c(i, 1), L::c(i, 2));
              if (wm >= 3) direct -= ls[i] * wall_term<L>(p, i, wm);
            }
          } else {
            ls[i] = (C)lam_in[i * N + n.at(L::c(i, 0), L::c(i, 1), L::c(i, 2))];
          }
        }
      }
      // forward state f(n)
      C f[L::Q];
      gather<L, S, G>(p, state, n, cls, f);
      C drho, j[3];
      moments<L>(f, drho, j);
      const C rho = C(1) + drho;
      const C inv = C(1) / rho;
      const C gamma = p.gamma ? p.gamma[n.cell] : C(1);
      C F[3];
      force_at(p, n.cell, F);
      C u[3], up[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        u[d] = (j[d] + C(0.5) * F[d]) * inv;
        up[d] = gamma * u[d];
      }
      // moments of mu_k = w_k lam*_k
      C m0 = C(0), m1[3] = {C(0), C(0), C(0)};
      C m2[3][3] = {{C(0), C(0), C(0)}, {C(0), C(0), C(0)}, {C(0), C(0), C(0)}};
      C lf = C(0);
#pragma unroll
      for (int k = 0; k < L::Q; ++k) {
        const C mu = (C)L::w(k) * ls[k];
        m0 += mu;
        lf += ls[k] * f[k];
#pragma unroll
        for (int a = 0; a < L::DIM; ++a) {
          if (L::c(k, a) == 1) m1[a] += mu;
          if (L::c(k, a) == -1) m1[a] -= mu;
#pragma unroll
          for (int b = a; b < L::DIM; ++b) {
            const int cc = L::c(k, a) * L::c(k, b);
            if (cc == 1) m2[a][b] += mu;
            if (cc == -1) m2[a][b] -= mu;
          }
        }
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < a; ++b) m2[a][b] = m2[b][a];
      const C om = p.omega;
      const C gf = C(1) - C(0.5) * om;
      const C om_odd = TRT ? p.omega_minus : om;  // relaxation rate of the odd part (m1)
      C m2u[3], m2F[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        m2u[a] = m2[a][0] * up[0] + m2[a][1] * up[1] + m2[a][2] * up[2];
        m2F[a] = m2[a][0] * F[0] + m2[a][1] * F[1] + m2[a][2] * F[2];
      }
      const C usq = up[0] * up[0] + up[1] * up[1] + up[2] * up[2];
      const C m1u = m1[0] * up[0] + m1[1] * up[1] + m1[2] * up[2];
      const C um2u = up[0] * m2u[0] + up[1] * m2u[1] + up[2] * m2u[2];
      // A - m0 (kept separately: the dL/domega term below needs it without the O(w) part)
      const C Aex = C(3) * m1u + C(4.5) * um2u - C(1.5) * m0 * usq;
      const C A = m0 + Aex;
      C B[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if constexpr (TRT)
          B[a] = rho * (om_odd * C(3) * m1[a] + om * (C(9) * m2u[a] - C(3) * m0 * up[a])) +
                 gf * (C(9) * m2F[a] - C(3) * m0 * F[a]);
        else
          B[a] = om * rho * (C(3) * m1[a] + C(9) * m2u[a] - C(3) * m0 * up[a]) +
                 gf * (C(9) * m2F[a] - C(3) * m0 * F[a]);
      }
      const C Bu = B[0] * u[0] + B[1] * u[1] + B[2] * u[2];
      const C gi = gamma * inv;
      C base;
      if constexpr (TRT)
        base = om * (m0 + C(4.5) * um2u - C(1.5) * m0 * usq) + om_odd * C(3) * m1u - gi * Bu + direct;
      else
        base = om * A - gi * Bu + direct;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        C Bc = C(0);
#pragma unroll
        for (int a = 0; a < L::DIM; ++a) {
          if (L::c(i, a) == 1) Bc += B[a];
          if (L::c(i, a) == -1) Bc -= B[a];
        }
        C own;
        if constexpr (TRT) {
          // lam*_i - omega+ (lam*_i + lam*_opp)/2 - omega- (lam*_i - lam*_opp)/2
          const C lo = ls[opp<L>(i)];
          own = ls[i] - om * (C(0.5) * (ls[i] + lo)) - om_odd * (C(0.5) * (ls[i] - lo));
        } else {
          own = (C(1) - om) * ls[i];
        }
        lam_out[i * N + n.cell] = (typename LambdaOf<S>::T)(own + base + gi * Bc);
      }
      if (dgamma) dgamma[n.cell] += (double)Bu;
      if (dforce) {
        // through u = (j + F/2)/rho (B gamma / (2 rho)) and the Guo source's own F;
        // TRT: the source's odd part (m1) carries 1 - omega-/2
        const C gf_odd = TRT ? C(1) - C(0.5) * om_odd : gf;
        const C hg = C(0.5) * gi;
#pragma unroll
        for (int a = 0; a < L::DIM; ++a)
          dforce[(size_t)a * p.ncell + n.cell] +=
              (double)(hg * B[a] + gf_odd * C(3) * m1[a] + gf * (C(9) * m2u[a] - C(3) * m0 * up[a]));
      }
      // dL/domega = sum_k lam*_k (feq_k - f_k) - G/2.  feq and f are both O(w) and
      // differ by the small non-equilibrium part, so the O(w) parts are removed
      // analytically before rounding: sum lam* (feq - w) = m0 drho + rho (A - m0)
      // and sum lam* (f - w) = lf (f stored shifted).
      const C m1F = m1[0] * F[0] + m1[1] * F[1] + m1[2] * F[2];
      const C uF = up[0] * F[0] + up[1] * F[1] + up[2] * F[2];
      const C uM2F = up[0] * m2F[0] + up[1] * m2F[1] + up[2] * m2F[2];
      if constexpr (TRT) {
        // the odd parts (m1 and the odd part of sum lam* f) move with omega- (omega)
        const C dwm = p.domega_minus;
        C lf_odd = C(0);
#pragma unroll
        for (int k = 1; k <= L::HALF; ++k)
          lf_odd += C(0.5) * (ls[k] - ls[k + L::HALF]) * (f[k] - f[k + L::HALF]);
        const C src_w = C(3) * dwm * m1F - C(3) * m0 * uF + C(9) * uM2F;
        const C Aex_w = C(3) * dwm * m1u + C(4.5) * um2u - C(1.5) * m0 * usq;
        sv[0] = m0 * drho + rho * Aex_w - (lf - lf_odd) - dwm * lf_odd - C(0.5) * src_w;
      } else {
        const C src_moment = C(3) * m1F - C(3) * m0 * uF + C(9) * uM2F;
        sv[0] = m0 * drho + rho * Aex - lf - C(0.5) * src_moment;
      }
    }
  }
  block_reduce_row(sv, partials + 8 * block_linear(), true);
}

// Objective (mean u[comp] over fluid cells of a plane) and its gradient seed
// lam^N_i(x) = (c_i[comp] - u[comp]) / (rho M) on those cells, 0 elsewhere.  With
// dforce: dL/dF(x) starts at the objective's own term 1/(2 rho M) on component comp
// of those cells (u = (j + F/2)/rho) and 0 elsewhere.
template <class L, class S, int G>
__global__ void __launch_bounds__(256) k_loss_seed(Params<typename Store<S>::C> p, const S* src, int axis,
                                                   int index, int comp, double inv_count,
                                                   typename LambdaOf<S>::T* lam, double* dforce,
                                                   double* partials) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const size_t N = (size_t)p.pitch;
  C sv[8] = {C(0), C(0), C(0), C(0), C(0), C(0), C(0), C(0)};
  if (x < p.nx && y < p.ny) {
    const Nbr n = make_nbr<L>(p, x, y, blockIdx.z);
    const int cls = p.all_fluid ? 1 : p.cls[n.cell];
    const int coord = axis == 0 ? x : (axis == 1 ? y : (int)blockIdx.z);
    if (cls != 0 && coord == index) {
      C f[L::Q];
      gather<L, S, G>(p, src, n, cls, f);
      C drho, j[3];
      moments<L>(f, drho, j);
      const C rho = C(1) + drho;
      C F[3];
      force_at(p, n.cell, F);
      const C jc = comp == 0 ? j[0] : (comp == 1 ? j[1] : j[2]);
      const C fc = C(0.5) * (comp == 0 ? F[0] : (comp == 1 ? F[1] : F[2]));
      const C uc = (jc + fc) / rho;
      sv[0] = uc;
      const C scale = (C)inv_count / rho;
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const int ci = comp == 0 ? L::c(i, 0) : (comp == 1 ? L::c(i, 1) : L::c(i, 2));
        lam[i * N + n.cell] = (typename LambdaOf<S>::T)(((C)ci - uc) * scale);
      }
      if (dforce) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
          dforce[(size_t)a * p.ncell + n.cell] = a == comp ? (double)(C(0.5) * scale) : 0.0;
      }
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) lam[i * N + n.cell] = 0;
      if (dforce) {
#pragma unroll
        for (int a = 0; a < 3; ++a) dforce[(size_t)a * p.ncell + n.cell] = 0.0;
      }
    }
  }
  block_reduce_row(sv, partials + 8 * block_linear(), false);
}

// Seed of the adjoint for the velocity misfit J = 1/2 sum over the fluid cells of
// the region of |u - u*|^2 (the objective of the guide's optimisation examples,
// section "optimization": domainIdentification3d, testFlowOpti3d), on the final
// state: lam_i = dJ/df_i = sum_a (u_a - u*_a) (c_ia - u_a) / rho, zero elsewhere.
// u_target is [d][cells] (FP64, canonical cell order), region a per-cell flag or
// nullptr (every fluid cell).  Partial row k = 0: J, k = 1: cells counted.
template <class L, class S, int G>
__global__ void __launch_bounds__(256) k_misfit_seed(Params<typename Store<S>::C> p, const S* src,
                                                     const double* u_target, const uint8_t* region,
                                                     typename LambdaOf<S>::T* lam, double* dforce,
                                                     double* partials) {
  using C = typename Store<S>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const size_t N = (size_t)p.pitch;
  C sv[8] = {C(0), C(0), C(0), C(0), C(0), C(0), C(0), C(0)};
  if (x < p.nx && y < p.ny) {
    const Nbr n = make_nbr<L>(p, x, y, blockIdx.z);
    const int cls = p.all_fluid ? 1 : p.cls[n.cell];
    if (cls != 0 && (region == nullptr || region[n.cell] != 0)) {
      C f[L::Q];
      gather<L, S, G>(p, src, n, cls, f);
      C drho, j[3];
      moments<L>(f, drho, j);
      const C rho = C(1) + drho;
      const C inv = C(1) / rho;
      C F[3];
      force_at(p, n.cell, F);
      C u[3], e[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        u[a] = (j[a] + C(0.5) * F[a]) * inv;
        e[a] = a < L::DIM ? u[a] - (C)u_target[(size_t)a * p.ncell + n.cell] : C(0);
        sv[0] += C(0.5) * e[a] * e[a];
      }
      sv[1] = C(1);
      // sum_a e_a (c_ia - u_a) / rho = (e . c_i - e . u) / rho
      const C eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const C ec = L::c(i, 0) * e[0] + L::c(i, 1) * e[1] + L::c(i, 2) * e[2];
        lam[i * N + n.cell] = (typename LambdaOf<S>::T)((ec - eu) * inv);
      }
      // dJ/dF(x) from the objective itself: e / (2 rho)
      if (dforce) {
#pragma unroll
        for (int a = 0; a < 3; ++a) dforce[(size_t)a * p.ncell + n.cell] = (double)(C(0.5) * e[a] * inv);
      }
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) lam[i * N + n.cell] = 0;
      if (dforce) {
#pragma unroll
        for (int a = 0; a < 3; ++a) dforce[(size_t)a * p.ncell + n.cell] = 0.0;
      }
    }
  }
  block_reduce_row(sv, partials + 8 * block_linear(), false);
}

}  // namespace olb

#include "olb_pair.cuh"
#include "olb_tma.cuh"

namespace olb {

// ---------------------------------------------------------------------------------
// Host launchers (dispatch run-time pattern choices to template instances).
// ---------------------------------------------------------------------------------
template <class L, class S>
struct Launch {
  using C = typename Store<S>::C;
  using T = typename LambdaOf<S>::T;

  static Params<C> params(const HostParams& h) {
    Params<C> p = to_params<C>(h);
    p.all_fluid = h.cls == nullptr ? 1 : 0;
    return p;
  }

  template <class PL>
  static void fill_planes(PL& pl, const void* src, void* dst, int pitch) {
    for (int i = 0; i < 19; ++i) {
      const int k = i < L::Q ? i : 0;
      pl.src[i] = static_cast<const S*>(src) + (size_t)k * pitch;
      pl.dst[i] = static_cast<S*>(dst) + (size_t)k * pitch;
    }
  }

  // Tile geometry of the TMA-fed pull step; false when the lattice does not fit it
  // (double storage, odd nx, a force field, nx > 512 or rows not a 16-byte multiple).
  static bool tma_geometry(const HostParams& h, TmaGeom& g) {
    if constexpr (std::is_same<S, double>::value) {
      return false;
    } else {
      if (!tma_setting("OLB_TMA", OLB_TMA) || !pairs_ok(h.nx) || h.ffield != nullptr || h.err == nullptr ||
          h.nx > 512)
        return false;
      const int e = (int)sizeof(S);
      const int nbx = h.nx <= 256 ? 1 : 2;
      const int bx = h.nx / nbx;
      // copy starts: x * elem a 16-byte multiple; shared destinations of the second
      // x box and of single rows (periodic y) 128-byte aligned
      if (nbx * bx != h.nx || (bx * e) % 16 != 0) return false;
      if (nbx == 2 && (bx * e) % 128 != 0) return false;
      if ((h.periodic & 2u) && (h.nx * e) % 128 != 0) return false;
      g.pairs = h.nx / 2;
      g.rows = 256 / g.pairs;
      if (g.rows < 1 || (nbx == 2 && g.rows != 1)) return false;
      g.nbx = nbx;
      g.bx = bx;
      const int ny_box = h.y1 - h.y0 + 1, nz_box = h.z1 - h.z0 + 1;
      if (ny_box < 1 || nz_box < 1) return false;
      g.tiles_y = (ny_box + g.rows - 1) / g.rows;
      g.ntiles = g.tiles_y * nz_box;
      g.stages = e == 4 ? tma_setting("OLB_TMA_STAGES32", OLB_TMA_STAGES32)
                        : tma_setting("OLB_TMA_STAGES16", OLB_TMA_STAGES16);
      if (g.stages < 2 || g.stages > kTmaMaxStages) return false;
      g.stage_bytes = (unsigned)(L::Q * g.rows * h.nx * e);
      g.box_slot = (unsigned)((g.rows * h.nx * e + 127) / 128 * 128);
      g.err = h.err;
      g.extra_tx = h.inject_extra_tx;
      g.warp_issue = tma_setting("OLB_TMA_WARP_ISSUE", OLB_TMA_WARP_ISSUE);
      g.release_early = tma_setting("OLB_TMA_RELEASE_EARLY", 0);
      // plain bulk copies need every row range 16-byte aligned (row bytes a 16-byte multiple) and one x box
      g.bulk1d = tma_setting("OLB_TMA_BULK1D", 0) && nbx == 1 && (h.nx * e) % 16 == 0;
      g.wait_ns = h.inject_extra_tx ? h.inject_wait_ns : kTmaWaitNs;
      return true;
    }
  }
  static size_t tma_smem(const TmaGeom& g) {
    return kTmaAlignSlack + kTmaBarrierBytes + (size_t)g.stages * L::Q * g.box_slot;
  }

  // Blocks of the persistent TMA grid: resident blocks per SM times SMs, at most one
  // per tile (0: the kernel cannot run with this shared memory).
  template <bool STATS, bool WALLS, bool TRT>
  static int tma_blocks(const TmaGeom& g, size_t smem) {
    if constexpr (std::is_same<S, double>::value) {
      return 0;
    } else {
      auto kernel = k_step_pair_tma<L, S, STATS, WALLS, TRT>;
      // per instance: the shared-memory size last configured and its occupancy
      static thread_local size_t set_bytes = 0;
      static thread_local int per_sm = 0, sms = 0;
      if (set_bytes != smem) {
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess) {
          cudaGetLastError();
          set_bytes = 0;
          return 0;
        }
        sms = device_sm_count();
        set_bytes = smem;
      }
      return std::min(per_sm * sms, g.ntiles);
    }
  }

  template <bool STATS, bool WALLS, bool TRT>
  static cudaError_t launch_tma(const HostParams& h, const TmaGeom& tg, int blocks, const void* src, void* dst,
                                double* partials) {
    if constexpr (std::is_same<S, double>::value) {
      return cudaErrorNotSupported;
    } else {
      // the tensor maps of the last few source buffers (a lattice alternates two)
      struct MapEntry {
        const void* src = nullptr;
        int nx = 0, ny = 0, nz = 0, pitch = 0, bx = 0, rows = 0;
        CUtensorMap tmain, trow;  // the type carries its 64-byte alignment
      };
      static thread_local MapEntry cache[4];
      static thread_local int next = 0;
      MapEntry* e = nullptr;
      for (auto& c : cache)
        if (c.src == src && c.nx == h.nx && c.ny == h.ny && c.nz == h.nz && c.pitch == h.pitch && c.bx == tg.bx &&
            c.rows == tg.rows)
          e = &c;
      if (!e) {
        e = &cache[next];
        next = (next + 1) % 4;
        const bool bf = std::is_same<S, __nv_bfloat16>::value;
        e->src = nullptr;
        if (!encode_population_map(&e->tmain, (int)sizeof(S), bf, src, h.nx, h.ny, h.nz, L::Q, h.pitch, tg.bx,
                                   tg.rows) ||
            !encode_population_map(&e->trow, (int)sizeof(S), bf, src, h.nx, h.ny, h.nz, L::Q, h.pitch, tg.bx, 1))
          return cudaErrorInvalidValue;
        e->src = src;
        e->nx = h.nx;
        e->ny = h.ny;
        e->nz = h.nz;
        e->pitch = h.pitch;
        e->bx = tg.bx;
        e->rows = tg.rows;
      }
      Params<float> p = params(h);
      Planes<S, WALLS> pl;
      if constexpr (WALLS) pl.lead = 0;
      fill_planes(pl, src, dst, h.pitch);
      return launch_step(k_step_pair_tma<L, S, STATS, WALLS, TRT>, dim3(blocks), dim3(256), tma_smem(tg), h.stream, p,
                         pl, e->tmain, e->trow, tg, partials);
    }
  }

  template <bool STATS, bool TRT>
  static int tma_blocks_for(const HostParams& h, const TmaGeom& tg) {
    const size_t smem = tma_smem(tg);
    if (h.cls == nullptr && !OLB_FORCE_WALLS) return tma_blocks<STATS, false, TRT>(tg, smem);
    return tma_blocks<STATS, true, TRT>(tg, smem);
  }

  // Rows of partial sums that step() with these patterns writes when stats is set.
  static int64_t step_rows(const HostParams& h, int gather, int scatter) {
    TmaGeom tg;
    if (gather == G_PULL && scatter == S_OWN && tma_geometry(h, tg)) {
      const int b = h.trt ? tma_blocks_for<true, true>(h, tg) : tma_blocks_for<true, false>(h, tg);
      if (b >= 1) return b;
    }
    return make_step_grid(h, !std::is_same<S, double>::value && pairs_ok(h.nx) && h.ffield == nullptr).blocks();
  }

  template <int G, int SC, bool STATS, bool TRT>
  static cudaError_t step_t(const HostParams& h, const void* src, void* dst, double* partials) {
    if constexpr (!std::is_same<S, double>::value && G == G_PULL && SC == S_OWN) {
      TmaGeom tg;
      if (tma_geometry(h, tg)) {
        const int blocks = tma_blocks_for<STATS, TRT>(h, tg);
        if (blocks >= 1) {
          if (h.cls == nullptr && !OLB_FORCE_WALLS)
            return launch_tma<STATS, false, TRT>(h, tg, blocks, src, dst, partials);
          return launch_tma<STATS, true, TRT>(h, tg, blocks, src, dst, partials);
        }
      }
    }
    if constexpr (!std::is_same<S, double>::value) {
      if (pairs_ok(h.nx) && h.ffield == nullptr) {  // the paired kernel takes a uniform force
        const StepGrid g = make_step_grid(h, true);
        Params<float> p = params(h);
        p.gx = g.gx;
        p.gy = g.gy;
        p.tile_shift = g.tile_shift;
        auto fill = [&](auto& pl) {
          for (int i = 0; i < 19; ++i) {
            const int k = i < L::Q ? i : 0;
            pl.src[i] = static_cast<const S*>(src) + (size_t)k * h.pitch;
            pl.dst[i] = static_cast<S*>(dst) + (size_t)k * h.pitch;
          }
        };
        if (h.cls == nullptr && !OLB_FORCE_WALLS) {  // all fluid, all periodic
          Planes<S, false> pl;
          fill(pl);
          return launch_step(k_step_pair<L, S, G, SC, STATS, false, TRT>, g.dims(), dim3(256), 0, h.stream, p, pl,
                             partials);
        }
        Planes<S, true> pl;
        pl.lead = 0;
        fill(pl);
        return launch_step(k_step_pair<L, S, G, SC, STATS, true, TRT>, g.dims(), dim3(256), 0, h.stream, p, pl,
                           partials);
      }
    }
    const StepGrid g = make_step_grid(h, false);
    return launch_step(k_step<L, S, G, SC, STATS, TRT>, g.dims(), dim3(256), 0, h.stream, params(h),
                       static_cast<const S*>(src), static_cast<S*>(dst), partials);
  }
  template <int G, int SC>
  static cudaError_t step_s(const HostParams& h, bool stats, const void* src, void* dst,
                            double* partials) {
    if (h.trt)
      return stats ? step_t<G, SC, true, true>(h, src, dst, partials)
                   : step_t<G, SC, false, true>(h, src, dst, partials);
    return stats ? step_t<G, SC, true, false>(h, src, dst, partials)
                 : step_t<G, SC, false, false>(h, src, dst, partials);
  }
  static cudaError_t step(const HostParams& h, int gather, int scatter, bool stats,
                          const void* src, void* dst, double* partials) {
    if (gather == G_OWN && scatter == S_OWN) return step_s<G_OWN, S_OWN>(h, stats, src, dst, partials);
    if (gather == G_PULL && scatter == S_OWN) return step_s<G_PULL, S_OWN>(h, stats, src, dst, partials);
    if (gather == G_PULL_SWAP && scatter == S_OWN)
      return step_s<G_PULL_SWAP, S_OWN>(h, stats, src, dst, partials);
    if (gather == G_OWN && scatter == S_OWN_SWAP)
      return step_s<G_OWN, S_OWN_SWAP>(h, stats, src, dst, partials);
    if (gather == G_PULL && scatter == S_OWN_SWAP)
      return step_s<G_PULL, S_OWN_SWAP>(h, stats, src, dst, partials);
    if (gather == G_PULL_SWAP && scatter == S_PUSH)
      return step_s<G_PULL_SWAP, S_PUSH>(h, stats, src, dst, partials);
    return cudaErrorInvalidValue;
  }

#define OLB_BY_GATHER(KERNEL, ...)                                                        \
  do {                                                                                    \
    Grid g = make_grid(h.nx, h.ny, h.nz);                                                 \
    if (gather == G_OWN)                                                                  \
      KERNEL<L, S, G_OWN><<<g.grid, g.block, 0, h.stream>>>(params(h), __VA_ARGS__);      \
    else if (gather == G_PULL)                                                            \
      KERNEL<L, S, G_PULL><<<g.grid, g.block, 0, h.stream>>>(params(h), __VA_ARGS__);     \
    else if (gather == G_PULL_SWAP)                                                       \
      KERNEL<L, S, G_PULL_SWAP><<<g.grid, g.block, 0, h.stream>>>(params(h), __VA_ARGS__); \
    else                                                                                  \
      return cudaErrorInvalidValue;                                                       \
    return cudaGetLastError();                                                            \
  } while (0)

  static cudaError_t to_f64(const HostParams& h, int gather, const void* src, double* f) {
    OLB_BY_GATHER(k_to_f64, static_cast<const S*>(src), f);
  }
  static cudaError_t moments(const HostParams& h, int gather, const void* src, double* rho,
                             double* u) {
    OLB_BY_GATHER(k_moments, static_cast<const S*>(src), rho, u);
  }
  static cudaError_t stats(const HostParams& h, int gather, const void* src, double* partials) {
    OLB_BY_GATHER(k_stats, static_cast<const S*>(src), partials);
  }
  static cudaError_t materialize(const HostParams& h, int gather, const void* src, void* dst) {
    OLB_BY_GATHER(k_materialize, static_cast<const S*>(src), static_cast<S*>(dst));
  }
  static cudaError_t loss_seed(const HostParams& h, int gather, const void* src, int axis,
                               int index, int comp, double inv_count, void* lam, double* dforce,
                               double* partials) {
    OLB_BY_GATHER(k_loss_seed, static_cast<const S*>(src), axis, index, comp, inv_count,
                  static_cast<T*>(lam), dforce, partials);
  }
  static cudaError_t misfit_seed(const HostParams& h, int gather, const void* src, const double* u_target,
                                 const uint8_t* region, void* lam, double* dforce, double* partials) {
    OLB_BY_GATHER(k_misfit_seed, static_cast<const S*>(src), u_target, region, static_cast<T*>(lam), dforce,
                  partials);
  }
#undef OLB_BY_GATHER
  template <bool TRT>
  static cudaError_t adjoint_t(const HostParams& h, int gather, const void* state, const void* lam_in,
                               void* lam_out, double* dgamma, double* dforce, double* partials) {
    Grid g = make_grid(h.nx, h.ny, h.nz);
    const S* st = static_cast<const S*>(state);
    const T* li = static_cast<const T*>(lam_in);
    T* lo = static_cast<T*>(lam_out);
    if (gather == G_OWN)
      return launch_step(k_adjoint<L, S, G_OWN, TRT>, g.grid, g.block, 0, h.stream, params(h), st, li, lo, dgamma,
                         dforce, partials);
    if (gather == G_PULL)
      return launch_step(k_adjoint<L, S, G_PULL, TRT>, g.grid, g.block, 0, h.stream, params(h), st, li, lo, dgamma,
                         dforce, partials);
    return cudaErrorInvalidValue;
  }
  static cudaError_t adjoint(const HostParams& h, int gather, const void* state,
                             const void* lam_in, void* lam_out, double* dgamma, double* dforce,
                             double* partials) {
    return h.trt ? adjoint_t<true>(h, gather, state, lam_in, lam_out, dgamma, dforce, partials)
                 : adjoint_t<false>(h, gather, state, lam_in, lam_out, dgamma, dforce, partials);
  }

  static cudaError_t from_f64(const HostParams& h, const double* f, void* dst) {
    Grid g = make_grid(h.nx, h.ny, h.nz);
    k_from_f64<L, S><<<g.grid, g.block, 0, h.stream>>>(params(h), f, static_cast<S*>(dst));
    return cudaGetLastError();
  }
  static cudaError_t init_eq(const HostParams& h, const double* rho, const double* u, void* dst) {
    Grid g = make_grid(h.nx, h.ny, h.nz);
    k_init_eq<L, S><<<g.grid, g.block, 0, h.stream>>>(params(h), rho, u, static_cast<S*>(dst));
    return cudaGetLastError();
  }
  static cudaError_t perturb(const HostParams& h, const double* df, void* dst) {
    Grid g = make_grid(h.nx, h.ny, h.nz);
    k_perturb<L, S><<<g.grid, g.block, 0, h.stream>>>(params(h), df, static_cast<S*>(dst));
    return cudaGetLastError();
  }

  static const KernelTable* table() {
    static const KernelTable t = {L::Q,       sizeof(S), sizeof(T), &step,    &step_rows, &to_f64,
                                  &moments,   &stats,    &from_f64, &init_eq, &perturb,
                                  &materialize, &adjoint, &loss_seed, &misfit_seed};
    return &t;
  }
};

}  // namespace olb
