// olb_internal.h -- host-side declarations shared by the ABI layer (olb_api.cu)
// and the per-lattice, per-storage-type kernel instantiation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace olb {

// State representations of a population buffer.
//   PRE     buffer holds f(t) at the cell's own slots (canonical layout)
//   POST    buffer holds f*(t-1) at the cell's own slots; f(t) = S f*(t-1) is
//           obtained by pulling from the neighbours (two-buffer pull scheme)
//   AA_ODD  buffer holds f*(t-1) with swapped slots (f*_i(x) at slot opp(i) of x),
//           the state between the two half-steps of the AA pattern
enum Repr { PRE = 0, POST = 1, AA_ODD = 2 };

// How a kernel reads f(t) of a cell and writes the post-collision values.
enum Gather { G_OWN = 0, G_PULL = 1, G_PULL_SWAP = 2 };
enum Scatter { S_OWN = 0, S_OWN_SWAP = 1, S_PUSH = 2 };

inline int gather_of(int repr) { return repr == PRE ? G_OWN : (repr == POST ? G_PULL : G_PULL_SWAP); }

// Everything a kernel needs to know about the lattice, in double precision;
// each instantiation unit converts it to its compute type.
struct HostParams {
  int nx, ny, nz;
  int ncell;
  int pitch;              // elements between population planes of stored fields
  unsigned periodic;
  const uint8_t* cls;     // per cell: 0 non-fluid, 1 fluid with only fluid links, 2 fluid with links to
                          // wall cells, 3 fluid with links leaving the domain (non-periodic edge)
  const uint32_t* wmask;  // per cell: bit i set when the pull source x - c_i is not a fluid cell
  const uint8_t* mat;     // material numbers
  const double* wall_u;   // [256][4] moving-wall velocities
  const float* wall_f;    // [256][20] 6 w_i (c_i . u_w) per material and direction, FP32
  int moving;             // a moving-wall material touches the fluid
  double omega;
  int trt;                // collision: 0 BGK, 1 TRT
  double omega_minus;     // TRT odd-part rate (from tau and the magic parameter)
  double domega_minus;    // d omega_minus / d omega at fixed magic parameter (BGK: 1)
  double force[3];
  int forced;
  const void* gamma;      // per-cell porosity in the compute type, or nullptr
  const void* ffield;     // per-cell force density [3][ncell] in the compute type, or nullptr
  const uint32_t* pmask;  // per cell: bit i set when x + c_i is a non-fluid cell of the lattice
  const uint32_t* word;   // per cell link word of the step kernel
  int outside_links;      // some fluid cell has a link leaving the domain
  int y0, y1, z0, z1;     // rows holding fluid cells: y in [y0, y1], z in [z0, z1]
  int az0, az1;           // active planes (a slab's interior): statistics count only these
  unsigned* err;          // device error word of the handle (set by kernels whose bounded waits ran out)
  unsigned inject_extra_tx;                // failure injection: bytes a TMA-fed step waits for beyond its copies
  unsigned long long inject_wait_ns;       // and the limit of its waits then
  cudaStream_t stream;
};

// Launch geometry: 2D blocks along (x, y), one z plane per grid z index.
struct Grid {
  dim3 block, grid;
  int64_t blocks() const { return (int64_t)grid.x * grid.y * grid.z; }
};
Grid make_grid(int nx, int ny, int nz);

// Grid of the step kernel: 1D over gx * gy * nz tiles of (1 << tile_shift) threads
// along x by (256 >> tile_shift) rows; a thread updates one cell, or two
// neighbouring cells (x0, x0 + 1) in the paired kernel.
struct StepGrid {
  int gx, gy, nz, tile_shift;
  int64_t blocks() const { return (int64_t)gx * gy * nz; }
  dim3 dims() const { return dim3(gx, gy, nz); }
};
StepGrid make_step_grid(int nx, int ny, int nz, bool pairs);
// Step grid restricted to the rows y in [y0, y1], z in [z0, z1].
StepGrid make_step_grid(const HostParams& h, bool pairs);
// The paired kernel runs for FP32-arithmetic storage types when nx is even.
#ifdef OLB_NO_PAIRS
inline bool pairs_ok(int) { return false; }
#else
inline bool pairs_ok(int nx) { return nx % 2 == 0; }
#endif

// Launchers of one (lattice, storage type) pair.  Each returns the CUDA error of
// the launch.  `partials` receives one row of 8 doubles per block (reductions).
struct KernelTable {
  int q;
  size_t state_elem;   // bytes per stored population
  size_t lambda_elem;  // bytes per adjoint population
  cudaError_t (*step)(const HostParams&, int gather, int scatter, bool stats, const void* src,
                      void* dst, double* partials);
  // rows of partial sums that step() with these patterns writes when stats is set
  int64_t (*step_rows)(const HostParams&, int gather, int scatter);
  cudaError_t (*to_f64)(const HostParams&, int gather, const void* src, double* f);
  cudaError_t (*moments)(const HostParams&, int gather, const void* src, double* rho, double* u);
  cudaError_t (*stats)(const HostParams&, int gather, const void* src, double* partials);
  cudaError_t (*from_f64)(const HostParams&, const double* f, void* dst);
  cudaError_t (*init_eq)(const HostParams&, const double* rho, const double* u, void* dst);
  cudaError_t (*perturb)(const HostParams&, const double* df, void* dst);
  cudaError_t (*materialize)(const HostParams&, int gather, const void* src, void* dst);
  // dgamma [cells] and dforce [3][cells] (either may be null) accumulate the
  // gradients; the seeds write lam^N and the objective's own dforce term.
  cudaError_t (*adjoint)(const HostParams&, int gather, const void* state, const void* lam_in,
                         void* lam_out, double* dgamma, double* dforce, double* partials);
  cudaError_t (*loss_seed)(const HostParams&, int gather, const void* src, int axis, int index,
                           int comp, double inv_count, void* lam, double* dforce, double* partials);
  cudaError_t (*misfit_seed)(const HostParams&, int gather, const void* src, const double* u_target,
                             const uint8_t* region, void* lam, double* dforce, double* partials);
};

// dtype: 0 f64, 1 f32, 2 f16 (shifted), 3 bf16 (shifted)
const KernelTable* table_d2q9_f64();
const KernelTable* table_d2q9_f32();
const KernelTable* table_d2q9_f16();
const KernelTable* table_d2q9_bf16();
const KernelTable* table_d3q19_f64();
const KernelTable* table_d3q19_f32();
const KernelTable* table_d3q19_f16();
const KernelTable* table_d3q19_bf16();

// Advection-diffusion lattice (D2Q5: q = 5, D3Q7: q = 7), kernels in olb_ade.cu.
struct AdeHost {
  int q;
  bool f64;               // storage and arithmetic in double (else float)
  int nx, ny, nz;
  int64_t ncell;
  double omega;
  double vu[3];           // uniform advection velocity (used when vf is null)
  const double* vf;       // per-cell velocity [3][ncell] or nullptr
  // boundaries (all null: every cell bulk, every axis periodic)
  const uint8_t* mat;     // per cell: 1 bulk, 0 no-flux wall, 2..255 Dirichlet cell
  const uint8_t* lmask;   // per cell: bit i when link i of a bulk cell hits a non-bulk cell or leaves the domain
  const double* wall_C;   // [256] Dirichlet values by material number
  unsigned periodic;      // axes that wrap (bit 0 x, 1 y, 2 z)
  cudaStream_t stream;
};
cudaError_t ade_step(const AdeHost& h, const void* src, void* dst);
cudaError_t ade_init(const AdeHost& h, const double* C, void* g);
cudaError_t ade_density(const AdeHost& h, const void* g, double* C);

// Host helpers of the TMA-fed step (olb_api.cu).  SM count of the current device,
// and a tiled tensor map (a CUtensorMap, 128 bytes at `map`) over the population
// planes of a buffer: dimensions (x, y, z, population), box (box_x, box_rows, 1, 1).
// Returns false when the driver does not provide the encoder or refuses the layout.
int device_sm_count();
// Tuning setting of the TMA-fed step: the environment variable `name` (read once)
// when set to an integer, else `fallback` (the compiled default).
int tma_setting(const char* name, int fallback);
bool encode_population_map(void* map, int elem_bytes, bool bf16, const void* base, int nx, int ny, int nz, int q,
                           int pitch, int box_x, int box_rows);

// Where a caller's array lives, seen from the current device: host memory
// (pageable or pinned), memory the current device can use (its own device
// allocations, or managed memory), or device memory of another GPU (refused by
// every entry point: the kernels would address it without peer access).
enum MemKind { MEM_HOST = 0, MEM_DEVICE = 1, MEM_OTHER_DEVICE = 2 };
MemKind mem_kind(const void* p);
// The classification from the pointer's attributes (memory type, the device that
// owns it) and the current device.
inline MemKind classify_memory(cudaMemoryType type, int owner_device, int current_device) {
  if (type == cudaMemoryTypeManaged) return MEM_DEVICE;
  if (type != cudaMemoryTypeDevice) return MEM_HOST;
  return owner_device == current_device ? MEM_DEVICE : MEM_OTHER_DEVICE;
}

// Record the message returned by olb_last_error() on this thread; returns code.
int set_error(int code, const char* msg);

// Sum the first `rows` rows of 8 doubles into out[8] (deterministic order).
cudaError_t reduce_partials(const double* partials, int64_t rows, double* out, cudaStream_t s);

}  // namespace olb
