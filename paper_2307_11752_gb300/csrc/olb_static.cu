// olb_static.cu -- olb_statistics_noalloc: the lattice statistics reduction for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is already
// reserved by another allocator (a framework's caching allocator that holds
// nearly all of the GPU), or a latency-sensitive caller for which the implicit
// device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.  This
// entry point computes the same statistics as olb_diagnostics, from a canonical
// population array the caller owns, and keeps its per-block partial sums in a
// fixed array in the library's own device memory instead of a buffer it
// allocates.  The array is a file-scope __device__ variable: every GPU that loads
// the library holds it (4 MiB) until the process exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "olb.h"
#include "olb_kernels.cuh"

namespace {

// Blocks of 256 cells whose partial sums fit in the fixed array: the largest
// lattice this entry point accepts has kMaxBlocks * 256 = 16,777,216 cells.
constexpr int kMaxBlocks = 65536;
constexpr int kMaxDevices = 64;

// One row of 8 partial sums per block (see olb::block_reduce_row).
static __device__ __align__(256) double g_partial_rows[kMaxBlocks * 8];

// Device address of g_partial_rows for each device, with the context it was
// looked up in (host code may not use the symbol itself: on the host it names a
// stand-in, not device memory).  A device reset destroys the context and the
// module with it; the next call then sees another current context and looks the
// address up again instead of using the stale one.
struct RowsAddress {
  CUcontext ctx = nullptr;
  double* addr = nullptr;
};
std::mutex g_setup_mu;
RowsAddress g_rows[kMaxDevices];
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;

int static_fail(int code, const char* msg) { return olb::set_error(code, msg); }

// Memory the current device can address (its own allocations or managed memory).
bool on_device(const void* p) { return olb::mem_kind(p) == olb::MEM_DEVICE; }

// Statistics of a canonical (unshifted, FP64) population array: per-cell
// contributions {rho - 1, j, |u|^2/2, |u|, non-finite, 1} over fluid cells,
// reduced per block into the row of the block.
template <class L>
__global__ void __launch_bounds__(256) k_stats_canonical(const double* __restrict__ f,
                                                         const uint8_t* __restrict__ mat, int64_t ncell,
                                                         double hfx, double hfy, double hfz, double* rows) {
  double sv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (c < ncell && (mat == nullptr || mat[c] == OLB_MAT_FLUID)) {
    double drho = -1.0, j[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const double v = f[i * ncell + c];
      drho += v;
#pragma unroll
      for (int a = 0; a < 3; ++a) j[a] += L::c(i, a) * v;
    }
    const double rho = 1.0 + drho;
    const double u[3] = {(j[0] + hfx) / rho, (j[1] + hfy) / rho, (j[2] + hfz) / rho};
    olb::stats_of(drho, j, u, sv);
  }
  olb::block_reduce_row(sv, rows + 8 * (int64_t)blockIdx.x, false);
}

// Sum the rows in a fixed order and write the 7 statistics of olb_diagnostics.
__global__ void k_stats_finish(const double* __restrict__ rows, int nrows, double* out) {
  __shared__ double sh[256][8];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int r = threadIdx.x; r < nrows; r += 256) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = (k == 5) ? fmax(acc[k], rows[8 * r + k]) : acc[k] + rows[8 * r + k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        sh[threadIdx.x][k] = (k == 5) ? fmax(sh[threadIdx.x][k], sh[threadIdx.x + s][k])
                                      : sh[threadIdx.x][k] + sh[threadIdx.x + s][k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sh[0][7] + sh[0][0];  // fluid cells + sum (rho - 1)
    out[1] = sh[0][1];
    out[2] = sh[0][2];
    out[3] = sh[0][3];
    out[4] = sh[0][4];
    out[5] = sh[0][5];
    out[6] = sh[0][6];
  }
}

// Device address of the partial-sum array on the current device, looked up with
// that device current the first time the device (in its current context) is
// seen, and reused afterwards.
int rows_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(OLB_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return static_fail(OLB_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_ctx_current) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return static_fail(OLB_ERR_CUDA, "cuCtxGetCurrent is not available from the driver");
    }
    g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
  }
  // null until the runtime has made the device's primary context current; the
  // symbol lookup below does that
  CUcontext ctx = nullptr;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  RowsAddress& r = g_rows[dev];
  if (!ctx || r.ctx != ctx || !r.addr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partial_rows);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return static_fail(OLB_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e) : "null symbol address");
    }
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return static_fail(OLB_ERR_CUDA, "no current CUDA context");
    r.ctx = ctx;
    r.addr = static_cast<double*>(p);
  }
  *out = r.addr;
  return OLB_OK;
}

}  // namespace

extern "C" {

int olb_statistics_noalloc(olb_descriptor d, int nx, int ny, int nz, const double* f,
                           const uint8_t* material, const double* force, double* out,
                           void* cuda_stream) {
  olb::set_error(OLB_OK, "");
  if (d != OLB_D2Q9 && d != OLB_D3Q19) return static_fail(OLB_ERR_ARG, "unknown descriptor");
  if (nx < 1 || ny < 1 || nz < 1 || (d == OLB_D2Q9 && nz != 1))
    return static_fail(OLB_ERR_ARG, "bad lattice size");
  const int64_t cells = (int64_t)nx * ny * nz;
  const int64_t blocks = (cells + 255) / 256;
  if (blocks > kMaxBlocks)
    return static_fail(OLB_ERR_ARG,
                       "lattice too large for olb_statistics_noalloc: at most 16,777,216 cells "
                       "(65,536 blocks of partial sums in its fixed scratch array)");
  if (!f || !out) return static_fail(OLB_ERR_ARG, "null populations or output");
  if (!on_device(f) || !on_device(out) || (material && !on_device(material)))
    return static_fail(OLB_ERR_ARG, "populations, material and output must be device memory of the current device");
  double* rows = nullptr;
  int rc = rows_address(&rows);
  if (rc) return rc;
  const double hf[3] = {force ? 0.5 * force[0] : 0.0, force ? 0.5 * force[1] : 0.0,
                        force ? 0.5 * force[2] : 0.0};
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (d == OLB_D2Q9)
    k_stats_canonical<olb::D2Q9><<<(unsigned)blocks, 256, 0, s>>>(f, material, cells, hf[0], hf[1], 0.0, rows);
  else
    k_stats_canonical<olb::D3Q19><<<(unsigned)blocks, 256, 0, s>>>(f, material, cells, hf[0], hf[1], hf[2], rows);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(OLB_ERR_CUDA, cudaGetErrorString(e));
  k_stats_finish<<<1, 256, 0, s>>>(rows, (int)blocks, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(OLB_ERR_CUDA, cudaGetErrorString(e));
  return OLB_OK;
}

}  // extern "C"
