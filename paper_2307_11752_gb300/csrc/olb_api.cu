// olb_api.cu -- the C ABI of include/olb.h: handle state, argument checks,
// host/device staging, representation bookkeeping and the checkpointed adjoint.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "olb.h"
#include "olb_internal.h"
#include "olb_kernels.cuh"

using namespace olb;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(OLB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define OLB_CUDA(call, what)                      \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

struct Provider {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*free_)(void*, void*) = nullptr;
  void* ctx = nullptr;
};
std::mutex g_provider_mu;
Provider g_provider;

// A device buffer owned by the library, released by the provider that made it.
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  Provider prov;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), prov(o.prov) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (!p) return;
    if (prov.alloc) {
      prov.free_(p, prov.ctx);
    } else {
      cudaFree(p);
    }
    p = nullptr;
    n = 0;
  }
  // Allocate `bytes` (no-op when already at least that large).  Returns OLB status.
  int reserve(size_t bytes) {
    if (p && n >= bytes) return OLB_OK;
    release();
    if (bytes == 0) bytes = 256;
    {
      std::lock_guard<std::mutex> lk(g_provider_mu);
      prov = g_provider;
    }
    if (prov.alloc) {
      p = prov.alloc(bytes, prov.ctx);
      if (!p) return fail(OLB_ERR_OOM, "allocator returned no memory for %zu bytes", bytes);
    } else {
      cudaError_t e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(OLB_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
      }
    }
    n = bytes;
    return OLB_OK;
  }
};

// Elements between two population planes.  Planes are padded so that their
// starting addresses do not share all low address bits (a power-of-two lattice,
// such as 128^3, would otherwise put the 19 loads of a warp at the same offset
// modulo 2^23 bytes), keeping 256-byte alignment of every plane.
// The step grid covers only the rows that hold fluid cells.
#ifndef OLB_FLUID_BOX
#define OLB_FLUID_BOX 1
#endif

#ifndef OLB_PLANE_PAD
#define OLB_PLANE_PAD 256
#endif
int plane_pitch(int64_t cells) {
  const int64_t aligned = (cells + 63) / 64 * 64;
  return (int)(aligned + OLB_PLANE_PAD);
}

const KernelTable* table_for(int d, int t) {
  static const KernelTable* (*tables[2][4])() = {
      {table_d2q9_f64, table_d2q9_f32, table_d2q9_f16, table_d2q9_bf16},
      {table_d3q19_f64, table_d3q19_f32, table_d3q19_f16, table_d3q19_bf16}};
  if (d < 0 || d > 1 || t < 0 || t > 3) return nullptr;
  return tables[d][t]();
}

// Makes `device` current for the scope and restores the previous device.
struct DeviceScope {
  int prev = -1, dev;
  explicit DeviceScope(int device) : dev(device) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceScope() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
};

// OLB_OK with *dev = (p is memory the current device can use), or OLB_ERR_ARG
// when p is device memory of another GPU.
int locate(const void* p, bool* dev, const char* what) {
  const MemKind k = mem_kind(p);
  if (k == MEM_OTHER_DEVICE) return fail(OLB_ERR_ARG, "%s is device memory of another GPU than the current one", what);
  *dev = k == MEM_DEVICE;
  return OLB_OK;
}

// Cell classes and link masks from the material numbers (same tables as the
// kernels).  cls: 0 non-fluid, 1 fluid with only fluid neighbours, 2 fluid with a
// non-fluid neighbour cell, 3 fluid with a link leaving the domain along a
// non-periodic axis.  wmask bit i: x - c_i is not fluid (or outside); pmask bit
// i: x + c_i is a non-fluid cell inside the domain.
template <class L>
void link_masks(int nx, int ny, int nz, unsigned periodic, const uint8_t* mat, uint8_t* cls,
                uint32_t* wmask, uint32_t* pmask, uint32_t* word, bool* moving, bool* any_wall,
                bool* outside_links) {
  *moving = false;
  *any_wall = false;
  *outside_links = false;
  const int e[3] = {nx, ny, nz};
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t c = ((int64_t)z * ny + y) * nx + x;
        wmask[c] = 0;
        pmask[c] = 0;
        word[c] = 0;
        if (mat[c] != OLB_MAT_FLUID) {
          cls[c] = 0;
          *any_wall = true;
          uint32_t nb = 0;  // bit k: x + c_k is a fluid cell
          for (int k = 1; k < L::Q; ++k) {
            int q[3] = {x + L::c(k, 0), y + L::c(k, 1), z + L::c(k, 2)};
            bool inside = true;
            for (int a = 0; a < 3; ++a) {
              if (q[a] < 0 || q[a] >= e[a]) {
                if (periodic & (1u << a)) q[a] = (q[a] + e[a]) % e[a];
                else inside = false;
              }
            }
            if (inside && mat[((int64_t)q[2] * ny + q[1]) * nx + q[0]] == OLB_MAT_FLUID) nb |= 1u << k;
          }
          word[c] = nb;
          continue;
        }
        bool moving_link = false, mixed = false;
        uint32_t wm = 0, pm = 0, mv = 0;
        int mm = -1;  // material of the moving links
        bool out = false;
        for (int i = 1; i < L::Q; ++i) {
          for (int sgn = -1; sgn <= 1; sgn += 2) {  // -1: pull source x - c_i, +1: push target x + c_i
            int q[3] = {x + sgn * L::c(i, 0), y + sgn * L::c(i, 1), z + sgn * L::c(i, 2)};
            bool inside = true;
            for (int a = 0; a < 3; ++a) {
              if (q[a] < 0 || q[a] >= e[a]) {
                if (periodic & (1u << a)) {
                  q[a] = (q[a] + e[a]) % e[a];
                } else {
                  inside = false;
                }
              }
            }
            const uint8_t nm = inside ? mat[((int64_t)q[2] * ny + q[1]) * nx + q[0]] : (uint8_t)OLB_MAT_VOID;
            if (!inside || nm != OLB_MAT_FLUID) {
              if (sgn < 0) wm |= 1u << i;
              if (sgn > 0 && inside) {
                pm |= 1u << i;
                if (nm >= 3) {
                  *moving = moving_link = true;
                  mv |= 1u << i;
                  if (mm >= 0 && mm != nm) mixed = true;
                  mm = nm;
                }
              }
              if (!inside) out = true;
            }
          }
        }
        wmask[c] = wm;
        pmask[c] = pm;
        uint32_t plane = 0;  // plane form of the moving links (see kWordPlaneShift)
        for (int ax = 0; moving_link && !mixed && ax < L::DIM && !plane; ++ax)
          for (int s = -1; s <= 1 && !plane; s += 2) {
            uint32_t sel = 0;
            for (int i = 1; i < L::Q; ++i)
              if (((pm >> i) & 1u) && L::c(i, ax) == s) sel |= 1u << i;
            if (sel == mv) plane = 1u + 2u * ax + (s > 0 ? 1u : 0u);
          }
        word[c] = kWordFluid | (moving_link ? kWordMoving : 0u) | pm |
                  (plane ? (plane << kWordPlaneShift) | ((uint32_t)mm << kWordMatShift) : 0u);
        cls[c] = out ? 3 : (wm ? 2 : 1);
        if (out) *outside_links = true;
        if (wm) *any_wall = true;
      }
}

}  // namespace

int olb::tma_setting(const char* name, int fallback) {
  static std::mutex mu;
  static std::vector<std::pair<std::string, int>> seen;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& kv : seen)
    if (kv.first == name) return kv.second;
  int v = fallback;
  if (const char* s = std::getenv(name)) {
    char* end = nullptr;
    const long x = std::strtol(s, &end, 10);
    if (end != s && *end == '\0') v = (int)x;
  }
  seen.emplace_back(name, v);
  return v;
}

int olb::device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

bool olb::encode_population_map(void* map, int elem_bytes, bool bf16, const void* base, int nx, int ny, int nz,
                                int q, int pitch, int box_x, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    cudaGetLastError();
  });
  if (!encode) return false;
  const CUtensorMapDataType type = elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)q};
  const cuuint64_t strides[3] = {(cuuint64_t)nx * elem_bytes, (cuuint64_t)nx * ny * elem_bytes,
                                 (cuuint64_t)pitch * elem_bytes};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_rows, 1, 1};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return encode(static_cast<CUtensorMap*>(map), type, 4, const_cast<void*>(base), dims, strides, box, estride,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

MemKind olb::mem_kind(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return MEM_HOST;
  }
  int dev = -1;
  if (a.type == cudaMemoryTypeDevice && cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MEM_OTHER_DEVICE;
  }
  return classify_memory(a.type, a.device, dev);
}

int olb::set_error(int code, const char* msg) {
  g_err = msg ? msg : "";
  return code;
}

// ---------------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------------
struct olb_lattice {
  int device = 0;  // the CUDA device the handle's buffers live on
  int desc = 0, dtype = 0, q = 0, dim = 0;
  int nx = 0, ny = 0, nz = 0, ncell = 0, pitch = 0;
  const KernelTable* kt = nullptr;
  cudaStream_t stream = nullptr;
  DevBuf buf[2];
  int cur = 0, repr = PRE, scheme = OLB_PULL;
  DevBuf mat, cls, wmask, pmask, word, wall_u, gamma, ffield, partials, out8, err;
  bool outside_links = false;
  int y0 = 0, y1 = 0, z0 = 0, z1 = 0;  // bounding rows of the fluid cells
  std::vector<uint8_t> h_mat;
  unsigned periodic = 0;
  bool all_fluid = false, moving = false;
  double h_wall[256][4];
  float h_wall_f[256][20];  // 6 w_i (c_i . u_w), computed in FP64 and rounded once
  double tau = 1.0, F[3] = {0.0, 0.0, 0.0};
  bool trt = false;     // collision operator: BGK, or TRT with magic parameter `magic`
  double magic = 0.25;
  bool has_gamma = false;
  bool has_ffield = false;  // a per-cell force density replaces the uniform force
  int za = 0, zb = 1 << 30;  // active planes (olb_set_active_planes); the others are halo planes
  unsigned inject_tx = 0;   // failure injection for the next step (olb_inject_stalled_copy)
  int64_t inject_ns = 0;
  int64_t time = 0, launches = 0;

  size_t state_bytes() const { return (size_t)q * pitch * kt->state_elem; }
  size_t compute_elem() const { return dtype == OLB_F64 ? sizeof(double) : sizeof(float); }

  HostParams params() const {
    HostParams p;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.ncell = ncell;
    p.pitch = pitch;
    p.periodic = periodic;
    p.cls = all_fluid ? nullptr : static_cast<const uint8_t*>(cls.p);
    p.wmask = static_cast<const uint32_t*>(wmask.p);
    p.mat = static_cast<const uint8_t*>(mat.p);
    p.wall_u = static_cast<const double*>(wall_u.p);
    p.wall_f = reinterpret_cast<const float*>(static_cast<const char*>(wall_u.p) + sizeof(h_wall));
    p.moving = moving ? 1 : 0;
    p.omega = 1.0 / tau;
    p.trt = trt ? 1 : 0;
    p.omega_minus = trt ? 1.0 / (magic / (tau - 0.5) + 0.5) : p.omega;
    // omega- = 1/(Lambda/a + 1/2) with a = 1/omega - 1/2: d omega-/d omega = -omega-^2 Lambda/(a omega)^2
    p.domega_minus = trt ? -p.omega_minus * p.omega_minus * magic / ((tau - 0.5) * (tau - 0.5) * p.omega * p.omega)
                         : 1.0;
    for (int a = 0; a < 3; ++a) p.force[a] = F[a];
    p.forced = (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0) ? 1 : 0;
    p.gamma = has_gamma ? gamma.p : nullptr;
    p.ffield = has_ffield ? ffield.p : nullptr;
    p.pmask = static_cast<const uint32_t*>(pmask.p);
    p.word = static_cast<const uint32_t*>(word.p);
    p.outside_links = outside_links ? 1 : 0;
    p.y0 = y0;
    p.y1 = y1;
    p.z0 = std::max(z0, za);
    p.z1 = std::min(z1, zb);
    p.az0 = za;
    p.az1 = std::min(zb, nz - 1);
    if (p.z1 < p.z0) p.z0 = p.z1 = std::max(0, std::min(za, nz - 1));  // no fluid in the active planes
    p.err = static_cast<unsigned*>(err.p);
    p.inject_extra_tx = inject_tx;
    p.inject_wait_ns = (unsigned long long)inject_ns;
    p.stream = stream;
    return p;
  }
  // blocks (= rows of partial sums) of the step kernel and of the per-cell kernels
  // rows of partial sums the step kernels may write (the largest of their grids)
  int64_t step_rows() const {
    const HostParams p = params();
    int64_t r = make_step_grid(p, dtype != OLB_F64 && pairs_ok(nx) && !has_ffield).blocks();
    return std::max(r, kt->step_rows(p, G_PULL, S_OWN));
  }
  int64_t cell_rows() const { return make_grid(nx, ny, nz).blocks(); }
  int64_t grid_blocks() const { return std::max(step_rows(), cell_rows()); }
};

namespace olb {

Grid make_grid(int nx, int ny, int nz) {
  Grid g;
  int bx = nx >= 256 ? 256 : ((nx + 31) / 32) * 32;
  int by = 256 / bx;
  if (by > ny) by = ny;
  if (by < 1) by = 1;
  g.block = dim3(bx, by, 1);
  g.grid = dim3((nx + bx - 1) / bx, (ny + by - 1) / by, nz);
  return g;
}

__global__ void k_reduce_rows(const double* __restrict__ rows, int64_t n, double* out) {
  __shared__ double sh[256][8];
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double v = rows[8 * r + k];
      acc[k] = (k == 5) ? fmax(acc[k], v) : acc[k] + v;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const double o = sh[threadIdx.x + s][k];
        sh[threadIdx.x][k] = (k == 5) ? fmax(sh[threadIdx.x][k], o) : sh[threadIdx.x][k] + o;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 8) out[threadIdx.x] = sh[0][threadIdx.x];
}

StepGrid make_step_grid(int nx, int ny, int nz, bool pairs) {
  StepGrid g;
  const int units = pairs ? nx / 2 : nx;  // threads needed along x
  int shift = 5;  // 32 .. 256 threads along x
  while (shift < 8 && (1 << shift) < units) ++shift;
  g.tile_shift = shift;
  const int rows = 256 >> shift;
  g.gx = (units + (1 << shift) - 1) >> shift;
  g.gy = (ny + rows - 1) / rows;
  g.nz = nz;
  return g;
}

StepGrid make_step_grid(const HostParams& h, bool pairs) {
  StepGrid g = make_step_grid(h.nx, h.y1 - h.y0 + 1, h.z1 - h.z0 + 1, pairs);
  return g;
}

cudaError_t reduce_partials(const double* partials, int64_t rows, double* out, cudaStream_t s) {
  k_reduce_rows<<<1, 256, 0, s>>>(partials, rows, out);
  return cudaGetLastError();
}

}  // namespace olb

namespace {

// The handle's device must be the current one: its kernels run on the current
// device and address the handle's buffers.
int check_device(int device) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (cur != device) return fail(OLB_ERR_ARG, "handle belongs to device %d but device %d is current", device, cur);
  return OLB_OK;
}

int check(olb_handle h) {
  if (!h) return fail(OLB_ERR_ARG, "null handle");
  g_err.clear();
  return check_device(h->device);
}

int launched(olb_handle h, cudaError_t e, const char* what) {
  if (e != cudaSuccess) return cuda_fail(e, what);
  h->launches++;
  return OLB_OK;
}

// Device view of a caller array of `bytes` bytes for reading.  Host memory is
// copied into h->stage (or `tmp`) on the handle's stream.
int input_view(olb_handle h, const void* p, size_t bytes, DevBuf& tmp, const void** out) {
  bool dev = false;
  int rc = locate(p, &dev, "input array");
  if (rc) return rc;
  if (dev) {
    *out = p;
    return OLB_OK;
  }
  rc = tmp.reserve(bytes);
  if (rc) return rc;
  OLB_CUDA(cudaMemcpyAsync(tmp.p, p, bytes, cudaMemcpyHostToDevice, h->stream), "staging copy");
  *out = tmp.p;
  return OLB_OK;
}

// Ensure the second population buffer exists.
int ensure_other(olb_handle h) {
  DevBuf& b = h->buf[1 - h->cur];
  if (b.p && b.n >= h->state_bytes()) return OLB_OK;
  int rc = b.reserve(h->state_bytes());
  if (rc) return rc;
  OLB_CUDA(cudaMemsetAsync(b.p, 0, h->state_bytes(), h->stream), "clear buffer");
  return OLB_OK;
}

int ensure_partials(olb_handle h, int64_t rows) {
  int rc = h->partials.reserve((size_t)rows * 8 * sizeof(double));
  if (rc) return rc;
  return h->out8.reserve(8 * sizeof(double));
}

// Bring the state into the canonical PRE representation.
int materialize(olb_handle h) {
  if (h->repr == PRE) return OLB_OK;
  int rc = ensure_other(h);
  if (rc) return rc;
  HostParams p = h->params();
  rc = launched(h, h->kt->materialize(p, gather_of(h->repr), h->buf[h->cur].p, h->buf[1 - h->cur].p),
                "materialize");
  if (rc) return rc;
  h->cur = 1 - h->cur;
  h->repr = PRE;
  return OLB_OK;
}

// One collide-and-stream step in the handle's scheme.  `rows`, when given,
// receives the number of partial-sum rows the step kernel wrote (stats).
int step_once(olb_handle h, bool stats, double* partials, int64_t* rows = nullptr) {
  HostParams p = h->params();
  const KernelTable* kt = h->kt;
  int rc;
  void* a = h->buf[h->cur].p;
  int g, sc;
  if (h->scheme == OLB_PULL) {
    sc = S_OWN;
    if (h->repr == PRE) {
      g = G_OWN;
      rc = launched(h, kt->step(p, g, sc, stats, a, a, partials), "step");
    } else {
      if ((rc = ensure_other(h))) return rc;
      void* b = h->buf[1 - h->cur].p;
      g = gather_of(h->repr);
      rc = launched(h, kt->step(p, g, sc, stats, a, b, partials), "step");
      if (!rc) h->cur = 1 - h->cur;
    }
    if (rc) return rc;
    h->repr = POST;
  } else {
    if (h->repr == PRE) {
      g = G_OWN;
      sc = S_OWN_SWAP;
      rc = launched(h, kt->step(p, g, sc, stats, a, a, partials), "step");
      if (rc) return rc;
      h->repr = AA_ODD;
    } else if (h->repr == AA_ODD) {
      g = G_PULL_SWAP;
      sc = S_PUSH;
      rc = launched(h, kt->step(p, g, sc, stats, a, a, partials), "step");
      if (rc) return rc;
      h->repr = PRE;
    } else {
      if ((rc = ensure_other(h))) return rc;
      void* b = h->buf[1 - h->cur].p;
      g = G_PULL;
      sc = S_OWN_SWAP;
      rc = launched(h, kt->step(p, g, sc, stats, a, b, partials), "step");
      if (rc) return rc;
      h->cur = 1 - h->cur;
      h->repr = AA_ODD;
    }
  }
  if (rows) *rows = kt->step_rows(p, g, sc);
  h->inject_tx = 0;  // an injection applies to one step
  h->time++;
  return OLB_OK;
}

// Reads and clears the handle's error word (synchronises the stream).
int check_error_word(olb_handle h) {
  unsigned v = 0;
  OLB_CUDA(cudaMemcpyAsync(&v, h->err.p, sizeof(v), cudaMemcpyDeviceToHost, h->stream), "error word read");
  OLB_CUDA(cudaStreamSynchronize(h->stream), "error word sync");
  if (v) {
    OLB_CUDA(cudaMemsetAsync(h->err.p, 0, sizeof(unsigned), h->stream), "error word clear");
    return fail(OLB_ERR_TIMEOUT, "a step kernel gave up waiting for its tile copies; the state is invalid");
  }
  return OLB_OK;
}

// Convert the 8 reduced statistics to the ABI's 7 and deliver them.
int deliver_stats(olb_handle h, double* out) {
  if (int rc = check_error_word(h)) return rc;
  double r[8];
  OLB_CUDA(cudaMemcpyAsync(r, h->out8.p, sizeof(r), cudaMemcpyDeviceToHost, h->stream), "stats copy");
  OLB_CUDA(cudaStreamSynchronize(h->stream), "stats sync");
  double o[7] = {r[7] + r[0], r[1], r[2], r[3], r[4], r[5], r[6]};
  bool dev = false;
  int rc = locate(out, &dev, "statistics output");
  if (rc) return rc;
  if (dev) {
    OLB_CUDA(cudaMemcpyAsync(out, o, sizeof(o), cudaMemcpyHostToDevice, h->stream), "stats out");
    OLB_CUDA(cudaStreamSynchronize(h->stream), "stats sync");
  } else {
    std::memcpy(out, o, sizeof(o));
  }
  if (o[6] > 0) return fail(OLB_ERR_NONFINITE, "%.0f cells hold non-finite populations", o[6]);
  return OLB_OK;
}

template <class L>
void wall_terms(olb_handle h) {
  for (int m = 0; m < 256; ++m) {
    const double* u = h->h_wall[m];
    for (int i = 0; i < 20; ++i) {
      if (i >= L::Q) {
        h->h_wall_f[m][i] = 0.0f;
        continue;
      }
      const double cu = L::c(i, 0) * u[0] + L::c(i, 1) * u[1] + L::c(i, 2) * u[2];
      h->h_wall_f[m][i] = (float)(6.0 * L::w(i) * cu);
    }
  }
}

int upload_wall(olb_handle h) {
  if (h->desc == OLB_D2Q9)
    wall_terms<D2Q9>(h);
  else
    wall_terms<D3Q19>(h);
  OLB_CUDA(cudaMemcpyAsync(h->wall_u.p, h->h_wall, sizeof(h->h_wall), cudaMemcpyHostToDevice,
                           h->stream),
           "wall velocity upload");
  OLB_CUDA(cudaMemcpyAsync(static_cast<char*>(h->wall_u.p) + sizeof(h->h_wall), h->h_wall_f,
                           sizeof(h->h_wall_f), cudaMemcpyHostToDevice, h->stream),
           "wall term upload");
  return OLB_OK;
}

// Forward sweep with checkpoints, objective seed, reverse sweep with segment
// recompute (olb_adjoint_run and olb_adjoint_run_misfit).  `seed` launches the
// kernel that writes lam^N = dL/df^N and the objective's partial sums (row 0);
// loss = loss_scale * (sum of row 0).
template <class Seed>
int adjoint_sweep(olb_handle h, int64_t n_steps, int64_t K, Seed&& seed, double loss_scale, double* loss,
                  double* dL_dgamma, double* dL_dtau, double* dL_dF = nullptr) {
  int rc;
  if (K > n_steps) K = n_steps;
  const int64_t nseg = (n_steps + K - 1) / K;
  const size_t sb = h->state_bytes();
  const size_t lb = (size_t)h->q * h->pitch * h->kt->lambda_elem;
  const int64_t rows = h->cell_rows();

  // buffers: checkpoints, segment slots 1..K-1, two adjoint fields, gradients
  std::vector<DevBuf> ckpt(nseg), seg(K);
  std::vector<int> ckpt_repr(nseg);
  DevBuf lam[2], dg, dF, part;
  for (auto& b : ckpt)
    if ((rc = b.reserve(sb))) return rc;
  for (int64_t k = 1; k < K; ++k)
    if ((rc = seg[k].reserve(sb))) return rc;
  if ((rc = lam[0].reserve(lb)) || (rc = lam[1].reserve(lb)) || (rc = dg.reserve((size_t)h->ncell * 8)) ||
      (rc = part.reserve((size_t)rows * 8 * sizeof(double))) || (rc = ensure_partials(h, h->grid_blocks())))
    return rc;
  if (dL_dF && (rc = dF.reserve((size_t)3 * h->ncell * sizeof(double)))) return rc;
  double* dFp = dL_dF ? static_cast<double*>(dF.p) : nullptr;
  if (h->repr == AA_ODD && (rc = materialize(h))) return rc;

  // forward sweep with checkpoints (pull pattern)
  const int saved_scheme = h->scheme;
  h->scheme = OLB_PULL;
  for (int64_t s = 0; s < nseg; ++s) {
    OLB_CUDA(cudaMemcpyAsync(ckpt[s].p, h->buf[h->cur].p, sb, cudaMemcpyDeviceToDevice, h->stream), "checkpoint");
    ckpt_repr[s] = h->repr;
    const int64_t ks = std::min<int64_t>(K, n_steps - s * K);
    for (int64_t k = 0; k < ks; ++k)
      if ((rc = step_once(h, false, nullptr))) {
        h->scheme = saved_scheme;
        return rc;
      }
  }
  h->scheme = saved_scheme;

  // objective and seed lam^N
  HostParams p = h->params();
  const KernelTable* kt = h->kt;
  double* partials = static_cast<double*>(h->partials.p);
  if ((rc = launched(h, seed(p, h->buf[h->cur].p, lam[0].p, dFp, partials), "loss"))) return rc;
  if ((rc = launched(h, reduce_partials(partials, rows, static_cast<double*>(h->out8.p), h->stream), "loss reduce")))
    return rc;
  double lsum[8];
  OLB_CUDA(cudaMemcpyAsync(lsum, h->out8.p, sizeof(lsum), cudaMemcpyDeviceToHost, h->stream), "loss copy");
  OLB_CUDA(cudaMemsetAsync(dg.p, 0, (size_t)h->ncell * 8, h->stream), "gradient clear");
  OLB_CUDA(cudaMemsetAsync(part.p, 0, (size_t)rows * 8 * sizeof(double), h->stream), "partials clear");

  // reverse sweep: recompute each segment, then step the adjoint back through it
  int li = 0;
  for (int64_t s = nseg - 1; s >= 0; --s) {
    const int64_t ks = std::min<int64_t>(K, n_steps - s * K);
    std::vector<const void*> slot(ks);
    std::vector<int> srepr(ks);
    slot[0] = ckpt[s].p;
    srepr[0] = ckpt_repr[s];
    for (int64_t k = 1; k < ks; ++k) {
      const int g = srepr[k - 1] == PRE ? G_OWN : G_PULL;
      if ((rc = launched(h, kt->step(p, g, S_OWN, false, slot[k - 1], seg[k].p, nullptr), "recompute"))) return rc;
      slot[k] = seg[k].p;
      srepr[k] = POST;
    }
    for (int64_t k = ks - 1; k >= 0; --k) {
      const int g = srepr[k] == PRE ? G_OWN : G_PULL;
      if ((rc = launched(h, kt->adjoint(p, g, slot[k], lam[li].p, lam[1 - li].p, static_cast<double*>(dg.p),
                                        dFp, static_cast<double*>(part.p)), "adjoint")))
        return rc;
      li = 1 - li;
    }
  }
  if ((rc = launched(h, reduce_partials(static_cast<double*>(part.p), rows, static_cast<double*>(h->out8.p), h->stream), "gradient reduce")))
    return rc;
  double gsum[8];
  OLB_CUDA(cudaMemcpyAsync(gsum, h->out8.p, sizeof(gsum), cudaMemcpyDeviceToHost, h->stream), "gradient copy");
  if (dL_dgamma) {
    OLB_CUDA(cudaMemcpyAsync(dL_dgamma, dg.p, (size_t)h->ncell * 8, cudaMemcpyDefault, h->stream), "gradient out");
  }
  if (dL_dF) {
    OLB_CUDA(cudaMemcpyAsync(dL_dF, dF.p, (size_t)3 * h->ncell * 8, cudaMemcpyDefault, h->stream),
             "force gradient out");
  }
  OLB_CUDA(cudaStreamSynchronize(h->stream), "adjoint sync");
  if (loss) *loss = lsum[0] * loss_scale;
  if (dL_dtau) *dL_dtau = -gsum[0] / (h->tau * h->tau);
  return OLB_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------
extern "C" {

const char* olb_last_error(void) { return g_err.c_str(); }

#define OLB_STR2(x) #x
#define OLB_STR(x) OLB_STR2(x)
const char* olb_build_info(void) {
  return "sm_103a step_min_blocks=" OLB_STR(OLB_STEP_MIN_BLOCKS) " pair_min_blocks=" OLB_STR(OLB_PAIR_MIN_BLOCKS) " pair16_min_blocks=" OLB_STR(OLB_PAIR16_MIN_BLOCKS) " pair16_walls_min_blocks=" OLB_STR(OLB_PAIR16_WALLS_MIN_BLOCKS) " ghost16=" OLB_STR(OLB_GHOST_FIRST16) OLB_STR(OLB_GHOST_COORDS16) " ghost32=" OLB_STR(OLB_GHOST_FIRST32) OLB_STR(OLB_GHOST_COORDS32)
         " solid_fill=" OLB_STR(OLB_SOLID_FILL) " xwall_pairs=" OLB_STR(OLB_XWALL_PAIRS) " fluid_box=" OLB_STR(OLB_FLUID_BOX) " pdl=" OLB_STR(OLB_PDL) " plane_pad=" OLB_STR(OLB_PLANE_PAD)
#ifdef OLB_NO_PAIRS
         " pairs=off"
#else
         " pairs=on"
#endif
      ;
}

int olb_set_allocator(void* (*alloc)(size_t, void*), void (*free_)(void*, void*), void* ctx) {
  std::lock_guard<std::mutex> lk(g_provider_mu);
  if (alloc && !free_) return fail(OLB_ERR_ARG, "allocator without a free function");
  g_provider.alloc = alloc;
  g_provider.free_ = alloc ? free_ : nullptr;
  g_provider.ctx = alloc ? ctx : nullptr;
  g_err.clear();
  return OLB_OK;
}

int olb_lattice_create(olb_descriptor d, int nx, int ny, int nz, olb_dtype t, olb_handle* out) {
  g_err.clear();
  if (!out) return fail(OLB_ERR_ARG, "null output handle pointer");
  *out = nullptr;
  const KernelTable* kt = table_for((int)d, (int)t);
  if (!kt) return fail(OLB_ERR_ARG, "unknown descriptor %d or dtype %d", (int)d, (int)t);
  if (nx < 1 || ny < 1 || nz < 1) return fail(OLB_ERR_ARG, "lattice sizes must be >= 1");
  if (d == OLB_D2Q9 && nz != 1) return fail(OLB_ERR_ARG, "D2Q9 requires nz == 1");
  const int64_t cells = (int64_t)nx * ny * nz;
  if (cells > 2147483647LL - 4096) return fail(OLB_ERR_ARG, "more than 2^31 - 4097 cells");
  if (nz > 65535) return fail(OLB_ERR_ARG, "nz > 65535");
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {  // no usable device: the first allocation reports it
    cudaGetLastError();
    device = 0;
  }
  olb_lattice* h = new olb_lattice();
  h->device = device;
  h->desc = (int)d;
  h->dtype = (int)t;
  h->kt = kt;
  h->q = kt->q;
  h->dim = d == OLB_D2Q9 ? 2 : 3;
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->ncell = (int)cells;
  h->pitch = plane_pitch(cells);
  std::memset(h->h_wall, 0, sizeof(h->h_wall));
  int rc;
  if ((rc = h->buf[0].reserve(h->state_bytes())) || (rc = h->mat.reserve(cells)) ||
      (rc = h->cls.reserve(cells)) || (rc = h->wmask.reserve(cells * 4)) || (rc = h->pmask.reserve(cells * 4)) ||
      (rc = h->word.reserve(cells * 4)) || (rc = h->err.reserve(sizeof(unsigned))) ||
      (rc = h->wall_u.reserve(sizeof(h->h_wall) + sizeof(h->h_wall_f))) ||
      (rc = ensure_partials(h, h->grid_blocks()))) {
    std::string msg = g_err;
    delete h;
    g_err = msg;
    return rc;
  }
  if (cudaMemset(h->err.p, 0, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(OLB_ERR_CUDA, "error word clear failed");
  }
  // all fluid, nothing periodic: every boundary link bounces back
  h->h_mat.assign(cells, OLB_MAT_FLUID);
  if ((rc = olb_set_material(h, h->h_mat.data(), 0)) || (rc = olb_init_equilibrium(h, nullptr, nullptr)) ||
      (rc = olb_synchronize(h))) {
    std::string msg = g_err;
    delete h;
    g_err = msg;
    return rc;
  }
  *out = h;
  return OLB_OK;
}

int olb_lattice_destroy(olb_handle h) {
  if (!h) return fail(OLB_ERR_ARG, "null handle");
  // release on the handle's own device, whichever device is current
  DeviceScope on(h->device);
  cudaStreamSynchronize(h->stream);
  delete h;
  g_err.clear();
  return OLB_OK;
}

int olb_set_stream(olb_handle h, void* cuda_stream) {
  int rc = check(h);
  if (rc) return rc;
  if (h->stream != (cudaStream_t)cuda_stream) {
    // order the new stream after everything queued on the old one
    OLB_CUDA(cudaStreamSynchronize(h->stream), "stream switch");
  }
  h->stream = (cudaStream_t)cuda_stream;
  return OLB_OK;
}

int olb_set_scheme(olb_handle h, olb_scheme s) {
  int rc = check(h);
  if (rc) return rc;
  if (s != OLB_PULL && s != OLB_AA) return fail(OLB_ERR_ARG, "unknown scheme %d", (int)s);
  h->scheme = (int)s;
  return OLB_OK;
}

int olb_set_material(olb_handle h, const uint8_t* material, unsigned periodic_mask) {
  int rc = check(h);
  if (rc) return rc;
  if (!material) return fail(OLB_ERR_ARG, "null material array");
  if (periodic_mask > 7) return fail(OLB_ERR_ARG, "periodic mask %u > 7", periodic_mask);
  if (h->dim == 2 && (periodic_mask & OLB_PERIODIC_Z))
    return fail(OLB_ERR_ARG, "z cannot be periodic on D2Q9");
  const size_t n = (size_t)h->ncell;
  std::vector<uint8_t> m(n);
  bool dev = false;
  if ((rc = locate(material, &dev, "material array"))) return rc;
  if (dev) {
    OLB_CUDA(cudaMemcpy(m.data(), material, n, cudaMemcpyDeviceToHost), "material read");
  } else {
    std::memcpy(m.data(), material, n);
  }
  // the current state is kept in the canonical form across the geometry change
  if ((rc = materialize(h))) return rc;
  std::vector<uint8_t> cls(n);
  std::vector<uint32_t> wm(n), pm(n), wd(n);
  bool moving = false, any_wall = false, outside_links = false;
  if (h->desc == OLB_D2Q9)
    link_masks<D2Q9>(h->nx, h->ny, h->nz, periodic_mask, m.data(), cls.data(), wm.data(), pm.data(), wd.data(),
                     &moving, &any_wall, &outside_links);
  else
    link_masks<D3Q19>(h->nx, h->ny, h->nz, periodic_mask, m.data(), cls.data(), wm.data(), pm.data(), wd.data(),
                      &moving, &any_wall, &outside_links);
  OLB_CUDA(cudaMemcpyAsync(h->mat.p, m.data(), n, cudaMemcpyHostToDevice, h->stream), "material upload");
  OLB_CUDA(cudaMemcpyAsync(h->cls.p, cls.data(), n, cudaMemcpyHostToDevice, h->stream), "class upload");
  OLB_CUDA(cudaMemcpyAsync(h->wmask.p, wm.data(), n * 4, cudaMemcpyHostToDevice, h->stream), "mask upload");
  OLB_CUDA(cudaMemcpyAsync(h->pmask.p, pm.data(), n * 4, cudaMemcpyHostToDevice, h->stream), "mask upload");
  OLB_CUDA(cudaMemcpyAsync(h->word.p, wd.data(), n * 4, cudaMemcpyHostToDevice, h->stream), "word upload");
  OLB_CUDA(cudaStreamSynchronize(h->stream), "material sync");
  h->h_mat.swap(m);
  h->periodic = periodic_mask;
  h->moving = moving;
  h->outside_links = outside_links;
  h->all_fluid = !any_wall;
  // rows that hold fluid cells; the step kernel skips the others (no cell there
  // is updated, and their bounce-back slots are written by fluid neighbours)
  int y0 = h->ny, y1 = -1, z0 = h->nz, z1 = -1;
  for (int z = 0; z < h->nz; ++z)
    for (int y = 0; y < h->ny; ++y) {
      const uint8_t* row = h->h_mat.data() + ((int64_t)z * h->ny + y) * h->nx;
      bool any = false;
      for (int x = 0; x < h->nx && !any; ++x) any = row[x] == OLB_MAT_FLUID;
      if (any) {
        y0 = std::min(y0, y);
        y1 = std::max(y1, y);
        z0 = std::min(z0, z);
        z1 = std::max(z1, z);
      }
    }
  if (y1 < 0 || OLB_SOLID_FILL || !OLB_FLUID_BOX) {  // no fluid cell, or solid cells written too: full grid
    y0 = 0;
    y1 = h->ny - 1;
    z0 = 0;
    z1 = h->nz - 1;
  }
  h->y0 = y0;
  h->y1 = y1;
  h->z0 = z0;
  h->z1 = z1;
  return upload_wall(h);
}

int olb_set_wall_velocity(olb_handle h, int material_id, const double u[3]) {
  int rc = check(h);
  if (rc) return rc;
  if (material_id < 3 || material_id > 255) return fail(OLB_ERR_ARG, "material %d is not a moving wall id", material_id);
  if (!u) return fail(OLB_ERR_ARG, "null velocity");
  for (int a = 0; a < 3; ++a) {
    if (!std::isfinite(u[a])) return fail(OLB_ERR_ARG, "non-finite wall velocity");
  }
  OLB_CUDA(cudaStreamSynchronize(h->stream), "wall sync");
  for (int a = 0; a < 3; ++a) h->h_wall[material_id][a] = (h->dim == 2 && a == 2) ? 0.0 : u[a];
  return upload_wall(h);
}

int olb_set_bgk(olb_handle h, double tau) {
  int rc = check(h);
  if (rc) return rc;
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(OLB_ERR_ARG, "tau must be > 1/2 (got %g)", tau);
  h->tau = tau;
  h->trt = false;
  return OLB_OK;
}

int olb_set_trt(olb_handle h, double tau, double magic) {
  int rc = check(h);
  if (rc) return rc;
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(OLB_ERR_ARG, "tau must be > 1/2 (got %g)", tau);
  if (!(magic > 0.0) || !std::isfinite(magic)) return fail(OLB_ERR_ARG, "magic parameter must be > 0 (got %g)", magic);
  h->tau = tau;
  h->magic = magic;
  h->trt = true;
  return OLB_OK;
}

int olb_set_force(olb_handle h, const double F[3]) {
  int rc = check(h);
  if (rc) return rc;
  if (!F) return fail(OLB_ERR_ARG, "null force");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(F[a])) return fail(OLB_ERR_ARG, "non-finite force");
  for (int a = 0; a < 3; ++a) h->F[a] = (h->dim == 2 && a == 2) ? 0.0 : F[a];
  return OLB_OK;
}

}  // extern "C"

namespace olb {
template <class C>
__global__ void k_convert_gamma(const double* __restrict__ in, C* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (C)in[i];
}
// out[i] = in[i] for i < zero_from, 0 for zero_from <= i < n.
template <class C>
__global__ void k_convert_field(const double* __restrict__ in, C* __restrict__ out, int64_t n, int64_t zero_from) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = i < zero_from ? (C)in[i] : C(0);
}
}  // namespace olb

extern "C" {

int olb_set_porosity(olb_handle h, const double* gamma) {
  int rc = check(h);
  if (rc) return rc;
  if (!gamma) {
    h->has_gamma = false;
    return OLB_OK;
  }
  DevBuf tmp;
  const void* g;
  if ((rc = input_view(h, gamma, (size_t)h->ncell * sizeof(double), tmp, &g))) return rc;
  if ((rc = h->gamma.reserve((size_t)h->ncell * h->compute_elem()))) return rc;
  const int nb = (h->ncell + 255) / 256;
  if (h->dtype == OLB_F64)
    k_convert_gamma<double><<<nb, 256, 0, h->stream>>>(static_cast<const double*>(g), static_cast<double*>(h->gamma.p), h->ncell);
  else
    k_convert_gamma<float><<<nb, 256, 0, h->stream>>>(static_cast<const double*>(g), static_cast<float*>(h->gamma.p), h->ncell);
  if ((rc = launched(h, cudaGetLastError(), "porosity"))) return rc;
  if (tmp.p) OLB_CUDA(cudaStreamSynchronize(h->stream), "porosity sync");
  h->has_gamma = true;
  return OLB_OK;
}

int olb_set_force_field(olb_handle h, const double* F) {
  int rc = check(h);
  if (rc) return rc;
  if (!F) {
    h->has_ffield = false;
    return OLB_OK;
  }
  DevBuf tmp;
  const void* src;
  if ((rc = input_view(h, F, (size_t)3 * h->ncell * sizeof(double), tmp, &src))) return rc;
  if ((rc = h->ffield.reserve((size_t)3 * h->ncell * h->compute_elem()))) return rc;
  const int64_t n = (int64_t)3 * h->ncell;
  const int nb = (int)((n + 255) / 256);
  const int64_t zero_from = h->dim == 2 ? (int64_t)2 * h->ncell : n;  // D2Q9: no z component
  if (h->dtype == OLB_F64)
    k_convert_field<double><<<nb, 256, 0, h->stream>>>(static_cast<const double*>(src),
                                                       static_cast<double*>(h->ffield.p), n, zero_from);
  else
    k_convert_field<float><<<nb, 256, 0, h->stream>>>(static_cast<const double*>(src),
                                                      static_cast<float*>(h->ffield.p), n, zero_from);
  if ((rc = launched(h, cudaGetLastError(), "force field"))) return rc;
  if (tmp.p) OLB_CUDA(cudaStreamSynchronize(h->stream), "force field sync");
  h->has_ffield = true;
  return OLB_OK;
}

int olb_init_equilibrium(olb_handle h, const double* rho, const double* u) {
  int rc = check(h);
  if (rc) return rc;
  DevBuf t1, t2;
  const void* r = nullptr;
  const void* v = nullptr;
  if (rho && (rc = input_view(h, rho, (size_t)h->ncell * sizeof(double), t1, &r))) return rc;
  if (u && (rc = input_view(h, u, (size_t)3 * h->ncell * sizeof(double), t2, &v))) return rc;
  HostParams p = h->params();
  if ((rc = launched(h, h->kt->init_eq(p, static_cast<const double*>(r), static_cast<const double*>(v), h->buf[h->cur].p), "init_equilibrium")))
    return rc;
  if (t1.p || t2.p) OLB_CUDA(cudaStreamSynchronize(h->stream), "init sync");
  h->repr = PRE;
  h->time = 0;
  return OLB_OK;
}

int olb_perturb_populations(olb_handle h, const double* df) {
  int rc = check(h);
  if (rc) return rc;
  if (!df) return fail(OLB_ERR_ARG, "null perturbation");
  DevBuf tmp;
  const void* d;
  if ((rc = input_view(h, df, (size_t)h->q * h->ncell * sizeof(double), tmp, &d))) return rc;
  if ((rc = materialize(h))) return rc;
  HostParams p = h->params();
  if ((rc = launched(h, h->kt->perturb(p, static_cast<const double*>(d), h->buf[h->cur].p), "perturb"))) return rc;
  if (tmp.p) OLB_CUDA(cudaStreamSynchronize(h->stream), "perturb sync");
  return OLB_OK;
}

int olb_set_populations(olb_handle h, const double* f) {
  int rc = check(h);
  if (rc) return rc;
  if (!f) return fail(OLB_ERR_ARG, "null populations");
  DevBuf tmp;
  const void* d;
  if ((rc = input_view(h, f, (size_t)h->q * h->ncell * sizeof(double), tmp, &d))) return rc;
  HostParams p = h->params();
  if ((rc = launched(h, h->kt->from_f64(p, static_cast<const double*>(d), h->buf[h->cur].p), "set_populations"))) return rc;
  if (tmp.p) OLB_CUDA(cudaStreamSynchronize(h->stream), "set sync");
  h->repr = PRE;
  h->time = 0;
  return OLB_OK;
}

int olb_get_populations(olb_handle h, double* f) {
  int rc = check(h);
  if (rc) return rc;
  if (!f) return fail(OLB_ERR_ARG, "null output");
  const size_t bytes = (size_t)h->q * h->ncell * sizeof(double);
  bool dev = false;
  if ((rc = locate(f, &dev, "population output"))) return rc;
  DevBuf tmp;
  if (!dev && (rc = tmp.reserve(bytes))) return rc;
  double* d = dev ? f : static_cast<double*>(tmp.p);
  HostParams p = h->params();
  if ((rc = launched(h, h->kt->to_f64(p, gather_of(h->repr), h->buf[h->cur].p, d), "get_populations"))) return rc;
  if (!dev) {
    OLB_CUDA(cudaMemcpyAsync(f, d, bytes, cudaMemcpyDeviceToHost, h->stream), "populations copy");
    OLB_CUDA(cudaStreamSynchronize(h->stream), "populations sync");
  }
  return OLB_OK;
}

int olb_step(olb_handle h, int64_t n) {
  int rc = check(h);
  if (rc) return rc;
  if (n < 0) return fail(OLB_ERR_ARG, "negative step count");
  for (int64_t s = 0; s < n; ++s)
    if ((rc = step_once(h, false, nullptr))) return rc;
  return OLB_OK;
}

int olb_step_stats(olb_handle h, int64_t n, double* out) {
  int rc = check(h);
  if (rc) return rc;
  if (n < 1) return fail(OLB_ERR_ARG, "olb_step_stats needs n >= 1");
  if (!out) return fail(OLB_ERR_ARG, "null output");
  if ((rc = ensure_partials(h, h->step_rows()))) return rc;
  for (int64_t s = 0; s + 1 < n; ++s)
    if ((rc = step_once(h, false, nullptr))) return rc;
  int64_t rows = 0;
  if ((rc = step_once(h, true, static_cast<double*>(h->partials.p), &rows))) return rc;
  if ((rc = launched(h, reduce_partials(static_cast<double*>(h->partials.p), rows, static_cast<double*>(h->out8.p), h->stream), "stats reduce")))
    return rc;
  return deliver_stats(h, out);
}

int olb_moments(olb_handle h, double* rho, double* u) {
  int rc = check(h);
  if (rc) return rc;
  if (!rho && !u) return OLB_OK;
  const size_t nr = (size_t)h->ncell * sizeof(double), nu = 3 * nr;
  bool dr = true, du = true;
  if (rho && (rc = locate(rho, &dr, "density output"))) return rc;
  if (u && (rc = locate(u, &du, "velocity output"))) return rc;
  DevBuf t1, t2;
  if (rho && !dr && (rc = t1.reserve(nr))) return rc;
  if (u && !du && (rc = t2.reserve(nu))) return rc;
  double* r = rho ? (dr ? rho : static_cast<double*>(t1.p)) : nullptr;
  double* v = u ? (du ? u : static_cast<double*>(t2.p)) : nullptr;
  HostParams p = h->params();
  if ((rc = launched(h, h->kt->moments(p, gather_of(h->repr), h->buf[h->cur].p, r, v), "moments"))) return rc;
  if (rho && !dr) OLB_CUDA(cudaMemcpyAsync(rho, r, nr, cudaMemcpyDeviceToHost, h->stream), "rho copy");
  if (u && !du) OLB_CUDA(cudaMemcpyAsync(u, v, nu, cudaMemcpyDeviceToHost, h->stream), "u copy");
  if (!dr || !du) OLB_CUDA(cudaStreamSynchronize(h->stream), "moments sync");
  return OLB_OK;
}

int olb_diagnostics(olb_handle h, double* out) {
  int rc = check(h);
  if (rc) return rc;
  if (!out) return fail(OLB_ERR_ARG, "null output");
  const int64_t rows = h->cell_rows();
  if ((rc = ensure_partials(h, rows))) return rc;
  HostParams p = h->params();
  if ((rc = launched(h, h->kt->stats(p, gather_of(h->repr), h->buf[h->cur].p, static_cast<double*>(h->partials.p)), "diagnostics")))
    return rc;
  if ((rc = launched(h, reduce_partials(static_cast<double*>(h->partials.p), rows, static_cast<double*>(h->out8.p), h->stream), "diagnostics reduce")))
    return rc;
  return deliver_stats(h, out);
}

int olb_synchronize(olb_handle h) {
  int rc = check(h);
  if (rc) return rc;
  OLB_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
  OLB_CUDA(cudaGetLastError(), "asynchronous error");
  return check_error_word(h);
}

}  // extern "C"

namespace olb {
// Slots of the populations that cross a z face of a slab, and the kernels that move
// one plane's worth of them between a lattice and a caller's buffer.
struct HaloSlots {
  int n;
  int s[8];
};

template <class E>
__global__ void k_halo_pack(const E* __restrict__ state, int64_t pitch, HaloSlots sl, int64_t plane_cells,
                            int64_t plane_offset, E* __restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= plane_cells) return;
#pragma unroll 1
  for (int k = 0; k < sl.n; ++k) out[k * plane_cells + c] = state[sl.s[k] * pitch + plane_offset + c];
}

// Only cells that are fluid receive: a wall cell of the halo plane holds in these
// slots the bounce-back values its own fluid neighbours stored there.
template <class E>
__global__ void k_halo_unpack(E* __restrict__ state, int64_t pitch, HaloSlots sl, int64_t plane_cells,
                              int64_t plane_offset, const uint8_t* __restrict__ mat, const E* __restrict__ in) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= plane_cells || mat[plane_offset + c] != 1) return;
#pragma unroll 1
  for (int k = 0; k < sl.n; ++k) state[sl.s[k] * pitch + plane_offset + c] = in[k * plane_cells + c];
}
}  // namespace olb

namespace {

// Populations with c_z == cz of the handle's lattice.
HaloSlots halo_slots(olb_handle h, int cz) {
  HaloSlots sl;
  sl.n = 0;
  for (int i = 0; i < h->q; ++i) {
    const int c = h->desc == OLB_D2Q9 ? D2Q9::c(i, 2) : D3Q19::c(i, 2);
    if (c == cz) sl.s[sl.n++] = i;
  }
  return sl;
}

// Checks shared by pack and unpack; plane index of the face.
int halo_check(olb_handle h, int face, const void* buf, bool unpack, int* plane) {
  if (h->desc != OLB_D3Q19) return fail(OLB_ERR_UNSUPPORTED, "slab halos are along z, on D3Q19");
  if (face != 0 && face != 1) return fail(OLB_ERR_ARG, "face must be 0 (low z) or 1 (high z)");
  if (!buf) return fail(OLB_ERR_ARG, "null halo buffer");
  bool dev = false;
  int rc = locate(buf, &dev, "halo buffer");
  if (rc) return rc;
  if (!dev) return fail(OLB_ERR_ARG, "the halo buffer must be device memory");
  if (h->za < 1 || h->zb > h->nz - 2)
    return fail(OLB_ERR_STATE, "set active planes that leave a halo plane on both z faces first");
  if (h->scheme != OLB_PULL || h->repr != POST)
    return fail(OLB_ERR_STATE, "halos are exchanged between pull steps (state after a step, pull scheme)");
  *plane = unpack ? (face == 0 ? h->za - 1 : h->zb + 1) : (face == 0 ? h->za : h->zb);
  return OLB_OK;
}

template <class E>
int halo_launch(olb_handle h, bool unpack, HaloSlots sl, int plane, void* buf) {
  const int64_t pc = (int64_t)h->nx * h->ny;
  const int nb = (int)((pc + 255) / 256);
  E* state = static_cast<E*>(h->buf[h->cur].p);
  if (unpack)
    k_halo_unpack<E><<<nb, 256, 0, h->stream>>>(state, h->pitch, sl, pc, plane * pc,
                                                 static_cast<const uint8_t*>(h->mat.p), static_cast<const E*>(buf));
  else
    k_halo_pack<E><<<nb, 256, 0, h->stream>>>(state, h->pitch, sl, pc, plane * pc, static_cast<E*>(buf));
  return launched(h, cudaGetLastError(), unpack ? "halo unpack" : "halo pack");
}

int halo_move(olb_handle h, int face, void* buf, bool unpack) {
  int plane = 0;
  int rc = halo_check(h, face, buf, unpack, &plane);
  if (rc) return rc;
  // the populations that leave through the face: c_z = -1 at the low face, +1 at the
  // high face; a halo plane receives those that enter: +1 at the low, -1 at the high
  const int cz = unpack ? (face == 0 ? 1 : -1) : (face == 0 ? -1 : 1);
  const HaloSlots sl = halo_slots(h, cz);
  switch (h->kt->state_elem) {
    case 8: return halo_launch<uint64_t>(h, unpack, sl, plane, buf);
    case 4: return halo_launch<uint32_t>(h, unpack, sl, plane, buf);
    default: return halo_launch<uint16_t>(h, unpack, sl, plane, buf);
  }
}

}  // namespace

extern "C" {

int olb_set_active_planes(olb_handle h, int z_first, int z_last) {
  int rc = check(h);
  if (rc) return rc;
  if (z_first == -1 && z_last == -1) {
    h->za = 0;
    h->zb = 1 << 30;
    return OLB_OK;
  }
  if (z_first < 0 || z_last >= h->nz || z_first > z_last) return fail(OLB_ERR_ARG, "bad plane range");
  h->za = z_first;
  h->zb = z_last;
  return OLB_OK;
}

int olb_halo_size(olb_handle h, int64_t* values, int* elem_bytes) {
  int rc = check(h);
  if (rc) return rc;
  if (h->desc != OLB_D3Q19) return fail(OLB_ERR_UNSUPPORTED, "slab halos are along z, on D3Q19");
  if (values) *values = (int64_t)halo_slots(h, 1).n * h->nx * h->ny;
  if (elem_bytes) *elem_bytes = (int)h->kt->state_elem;
  return OLB_OK;
}

int olb_halo_pack(olb_handle h, int face, void* buf) {
  int rc = check(h);
  if (rc) return rc;
  return halo_move(h, face, buf, false);
}

int olb_halo_unpack(olb_handle h, int face, const void* buf) {
  int rc = check(h);
  if (rc) return rc;
  return halo_move(h, face, const_cast<void*>(buf), true);
}

int olb_inject_stalled_copy(olb_handle h, unsigned extra_bytes, int64_t wait_ns) {
  int rc = check(h);
  if (rc) return rc;
  if (extra_bytes > 65536u) return fail(OLB_ERR_ARG, "extra_bytes above 65536");
  if (extra_bytes && (wait_ns < 1000000 || wait_ns > 5000000000LL))
    return fail(OLB_ERR_ARG, "wait_ns outside [1 ms, 5 s]");
  h->inject_tx = extra_bytes;
  h->inject_ns = wait_ns;
  return OLB_OK;
}

int olb_counters(olb_handle h, int64_t* time, int64_t* kernel_launches) {
  int rc = check(h);
  if (rc) return rc;
  if (time) *time = h->time;
  if (kernel_launches) *kernel_launches = h->launches;
  return OLB_OK;
}

}  // extern "C"

namespace {

// The checkpointed adjoint of the plane-mean objective (obj) or of the velocity
// misfit (u_target, region), with every gradient output (any may be null).
int adjoint_plane(olb_handle h, int64_t n_steps, int64_t K, const olb_objective* obj, double* loss,
                  double* dL_dgamma, double* dL_dtau, double* dL_dF) {
  if (n_steps < 1 || K < 1) return fail(OLB_ERR_ARG, "n_steps and checkpoint_every must be >= 1");
  if (!obj || obj->plane_axis < 0 || obj->plane_axis >= h->dim || obj->component < 0 || obj->component >= h->dim)
    return fail(OLB_ERR_ARG, "bad objective");
  const int ext[3] = {h->nx, h->ny, h->nz};
  if (obj->plane_index < 0 || obj->plane_index >= ext[obj->plane_axis])
    return fail(OLB_ERR_ARG, "objective plane index out of range");
  int64_t count = 0;
  for (int z = 0; z < h->nz; ++z)
    for (int y = 0; y < h->ny; ++y)
      for (int x = 0; x < h->nx; ++x) {
        const int c[3] = {x, y, z};
        if (c[obj->plane_axis] == obj->plane_index && h->h_mat[((int64_t)z * h->ny + y) * h->nx + x] == OLB_MAT_FLUID)
          ++count;
      }
  if (count == 0) return fail(OLB_ERR_ARG, "objective plane holds no fluid cell");
  const double inv_count = 1.0 / (double)count;
  auto seed = [&](const HostParams& p, const void* state, void* lam0, double* dforce, double* partials) {
    return h->kt->loss_seed(p, gather_of(h->repr), state, obj->plane_axis, obj->plane_index, obj->component,
                            inv_count, lam0, dforce, partials);
  };
  return adjoint_sweep(h, n_steps, K, seed, inv_count, loss, dL_dgamma, dL_dtau, dL_dF);
}

int adjoint_misfit(olb_handle h, int64_t n_steps, int64_t K, const double* u_target, const uint8_t* region,
                   double* loss, double* dL_dgamma, double* dL_dtau, double* dL_dF) {
  int rc;
  if (n_steps < 1 || K < 1) return fail(OLB_ERR_ARG, "n_steps and checkpoint_every must be >= 1");
  if (!u_target) return fail(OLB_ERR_ARG, "null target velocity");
  const size_t n = (size_t)h->ncell;
  // the region on the host, to count its fluid cells before any work is queued
  std::vector<uint8_t> reg_host;
  if (region) {
    reg_host.resize(n);
    OLB_CUDA(cudaMemcpyAsync(reg_host.data(), region, n, cudaMemcpyDefault, h->stream), "region copy");
    OLB_CUDA(cudaStreamSynchronize(h->stream), "region sync");
  }
  int64_t count = 0;
  for (size_t c = 0; c < n; ++c)
    if (h->h_mat[c] == OLB_MAT_FLUID && (!region || reg_host[c] != 0)) ++count;
  if (count == 0) return fail(OLB_ERR_ARG, "objective region holds no fluid cell");
  DevBuf ut_tmp, reg_tmp;
  const void* ut = nullptr;
  const void* rg = nullptr;
  if ((rc = input_view(h, u_target, 3 * n * sizeof(double), ut_tmp, &ut))) return rc;
  if (region && (rc = input_view(h, region, n, reg_tmp, &rg))) return rc;
  auto seed = [&](const HostParams& p, const void* state, void* lam0, double* dforce, double* partials) {
    return h->kt->misfit_seed(p, gather_of(h->repr), state, static_cast<const double*>(ut),
                              static_cast<const uint8_t*>(rg), lam0, dforce, partials);
  };
  return adjoint_sweep(h, n_steps, K, seed, 1.0, loss, dL_dgamma, dL_dtau, dL_dF);
}

}  // namespace

extern "C" {

int olb_adjoint_run(olb_handle h, int64_t n_steps, int64_t K, const olb_objective* obj,
                    double* loss, double* dL_dgamma, double* dL_dtau) {
  int rc = check(h);
  if (rc) return rc;
  return adjoint_plane(h, n_steps, K, obj, loss, dL_dgamma, dL_dtau, nullptr);
}

int olb_adjoint_run_misfit(olb_handle h, int64_t n_steps, int64_t K, const double* u_target,
                           const uint8_t* region, double* loss, double* dL_dgamma, double* dL_dtau) {
  int rc = check(h);
  if (rc) return rc;
  return adjoint_misfit(h, n_steps, K, u_target, region, loss, dL_dgamma, dL_dtau, nullptr);
}

int olb_adjoint_gradients(olb_handle h, int64_t n_steps, int64_t K, const olb_objective* obj,
                          const double* u_target, const uint8_t* region, olb_gradients* out) {
  int rc = check(h);
  if (rc) return rc;
  if (!out) return fail(OLB_ERR_ARG, "null gradient outputs");
  if ((obj != nullptr) == (u_target != nullptr))
    return fail(OLB_ERR_ARG, "give either a plane objective or a target velocity, not both or neither");
  if (obj) return adjoint_plane(h, n_steps, K, obj, out->loss, out->dL_dgamma, out->dL_dtau, out->dL_dF);
  return adjoint_misfit(h, n_steps, K, u_target, region, out->loss, out->dL_dgamma, out->dL_dtau, out->dL_dF);
}

// ---------------------------------------------------------------------------------
// Advection-diffusion lattice
// ---------------------------------------------------------------------------------
}  // extern "C"

struct olb_ade {
  int device = 0;  // the CUDA device the handle's buffers live on
  int q = 0, dtype = 0;
  int nx = 0, ny = 0, nz = 0;
  int64_t ncell = 0;
  cudaStream_t stream = nullptr;
  DevBuf buf[2], vfield, stage, mat, lmask, wallC;
  int cur = 0;
  double tau = 1.0;
  double vu[3] = {0.0, 0.0, 0.0};
  bool has_vfield = false;
  bool has_bc = false;     // olb_ade_set_material was called
  unsigned periodic = 7u;
  size_t elem() const { return dtype == OLB_F64 ? sizeof(double) : sizeof(float); }
  size_t state_bytes() const { return (size_t)q * ncell * elem(); }
  AdeHost host() const {
    AdeHost a;
    a.q = q;
    a.f64 = dtype == OLB_F64;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.ncell = ncell;
    a.omega = 1.0 / tau;
    for (int k = 0; k < 3; ++k) a.vu[k] = vu[k];
    a.vf = has_vfield ? static_cast<const double*>(vfield.p) : nullptr;
    a.mat = has_bc ? static_cast<const uint8_t*>(mat.p) : nullptr;
    a.lmask = has_bc ? static_cast<const uint8_t*>(lmask.p) : nullptr;
    a.wall_C = has_bc ? static_cast<const double*>(wallC.p) : nullptr;
    a.periodic = has_bc ? periodic : 7u;
    a.stream = stream;
    return a;
  }
};

namespace {

int ade_check(olb_ade_handle h) {
  if (!h) return fail(OLB_ERR_ARG, "null advection-diffusion handle");
  return check_device(h->device);
}

// Device view of `bytes` bytes at p (copied into `tmp` when p is host memory).
int ade_input(olb_ade_handle h, const void* p, size_t bytes, DevBuf& tmp, const void** out) {
  bool dev = false;
  int rc = locate(p, &dev, "input array");
  if (rc) return rc;
  if (dev) {
    *out = p;
    return OLB_OK;
  }
  rc = tmp.reserve(bytes);
  if (rc) return rc;
  OLB_CUDA(cudaMemcpyAsync(tmp.p, p, bytes, cudaMemcpyHostToDevice, h->stream), "staging copy");
  *out = tmp.p;
  return OLB_OK;
}

}  // namespace

extern "C" {

int olb_ade_create(int descriptor, int nx, int ny, int nz, int dtype, olb_ade_handle* out) {
  if (!out) return fail(OLB_ERR_ARG, "null output handle");
  *out = nullptr;
  if (descriptor != OLB_D2Q5 && descriptor != OLB_D3Q7) return fail(OLB_ERR_ARG, "descriptor must be D2Q5 or D3Q7");
  if (dtype != OLB_F64 && dtype != OLB_F32) return fail(OLB_ERR_ARG, "advection-diffusion storage is F64 or F32");
  if (nx < 1 || ny < 1 || nz < 1) return fail(OLB_ERR_ARG, "lattice extents must be >= 1");
  if (descriptor == OLB_D2Q5 && nz != 1) return fail(OLB_ERR_ARG, "D2Q5 needs nz == 1");
  const int64_t cells = (int64_t)nx * ny * nz;
  if (cells > ((int64_t)1 << 31) / 8) return fail(OLB_ERR_ARG, "lattice too large (%lld cells)", (long long)cells);
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {  // no usable device: the first allocation reports it
    cudaGetLastError();
    device = 0;
  }
  olb_ade* h = new olb_ade();
  h->device = device;
  h->q = descriptor == OLB_D2Q5 ? 5 : 7;
  h->dtype = dtype;
  h->nx = nx;
  h->ny = ny;
  h->nz = nz;
  h->ncell = cells;
  int rc;
  if ((rc = h->buf[0].reserve(h->state_bytes())) || (rc = h->buf[1].reserve(h->state_bytes()))) {
    std::string msg = g_err;
    delete h;
    g_err = msg;
    return rc;
  }
  *out = h;
  return OLB_OK;
}

int olb_ade_destroy(olb_ade_handle h) {
  if (!h) return fail(OLB_ERR_ARG, "null advection-diffusion handle");
  DeviceScope on(h->device);
  cudaStreamSynchronize(h->stream);
  delete h;
  return OLB_OK;
}

int olb_ade_set_stream(olb_ade_handle h, void* stream) {
  int rc = ade_check(h);
  if (rc) return rc;
  h->stream = static_cast<cudaStream_t>(stream);
  return OLB_OK;
}

int olb_ade_set_tau(olb_ade_handle h, double tau) {
  int rc = ade_check(h);
  if (rc) return rc;
  if (!(tau > 0.5) || !std::isfinite(tau)) return fail(OLB_ERR_ARG, "tau must be > 1/2 (got %g)", tau);
  h->tau = tau;
  return OLB_OK;
}

int olb_ade_set_velocity(olb_ade_handle h, const double v[3], const double* v_field) {
  int rc = ade_check(h);
  if (rc) return rc;
  if (!v && !v_field) return fail(OLB_ERR_ARG, "no velocity given");
  if (v) {
    for (int a = 0; a < 3; ++a)
      if (!std::isfinite(v[a])) return fail(OLB_ERR_ARG, "non-finite velocity");
  }
  if (v_field) {
    const size_t bytes = 3 * (size_t)h->ncell * sizeof(double);
    if ((rc = h->vfield.reserve(bytes))) return rc;
    OLB_CUDA(cudaMemcpyAsync(h->vfield.p, v_field, bytes, cudaMemcpyDefault, h->stream), "velocity copy");
    OLB_CUDA(cudaStreamSynchronize(h->stream), "velocity sync");
    h->has_vfield = true;
  } else {
    for (int a = 0; a < 3; ++a) h->vu[a] = (h->q == 5 && a == 2) ? 0.0 : v[a];
    h->has_vfield = false;
  }
  return OLB_OK;
}

int olb_ade_set_material(olb_ade_handle h, const uint8_t* material, unsigned periodic_mask, const double* wall_C) {
  int rc = ade_check(h);
  if (rc) return rc;
  if (!material) return fail(OLB_ERR_ARG, "null material array");
  if (periodic_mask > 7 || (h->q == 5 && (periodic_mask & 4u))) return fail(OLB_ERR_ARG, "bad periodic mask %u", periodic_mask);
  const size_t n = (size_t)h->ncell;
  std::vector<uint8_t> m(n), lm(n);
  OLB_CUDA(cudaMemcpyAsync(m.data(), material, n, cudaMemcpyDefault, h->stream), "material read");
  OLB_CUDA(cudaStreamSynchronize(h->stream), "material sync");
  double wc[256] = {0.0};
  bool dirichlet = false;
  for (size_t c = 0; c < n; ++c) dirichlet |= m[c] >= 2;
  if (dirichlet && !wall_C) return fail(OLB_ERR_ARG, "Dirichlet cells (material >= 2) need wall_C");
  if (wall_C) {
    for (int k = 0; k < 256; ++k) {
      wc[k] = wall_C[k];
      if (!std::isfinite(wc[k])) return fail(OLB_ERR_ARG, "non-finite wall value");
    }
  }
  // per bulk cell: bit i when x + c_i is not a bulk cell or lies outside a non-periodic face
  static const int c5[5][3] = {{0, 0, 0}, {-1, 0, 0}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}};
  static const int c7[7][3] = {{0, 0, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  const int e[3] = {h->nx, h->ny, h->nz};
  for (int z = 0; z < h->nz; ++z)
    for (int y = 0; y < h->ny; ++y)
      for (int x = 0; x < h->nx; ++x) {
        const size_t c = ((size_t)z * h->ny + y) * h->nx + x;
        unsigned bits = 0;
        if (m[c] == 1) {
          for (int i = 1; i < h->q; ++i) {
            const int* ci = h->q == 5 ? c5[i] : c7[i];
            int p[3] = {x + ci[0], y + ci[1], z + ci[2]};
            bool inside = true;
            for (int a = 0; a < 3; ++a)
              if (p[a] < 0 || p[a] >= e[a]) {
                if (periodic_mask & (1u << a)) p[a] = (p[a] + e[a]) % e[a];
                else inside = false;
              }
            if (!inside || m[((size_t)p[2] * h->ny + p[1]) * h->nx + p[0]] != 1) bits |= 1u << i;
          }
        }
        lm[c] = (uint8_t)bits;
      }
  if ((rc = h->mat.reserve(n)) || (rc = h->lmask.reserve(n)) || (rc = h->wallC.reserve(sizeof(wc)))) return rc;
  OLB_CUDA(cudaMemcpyAsync(h->mat.p, m.data(), n, cudaMemcpyHostToDevice, h->stream), "material upload");
  OLB_CUDA(cudaMemcpyAsync(h->lmask.p, lm.data(), n, cudaMemcpyHostToDevice, h->stream), "mask upload");
  OLB_CUDA(cudaMemcpyAsync(h->wallC.p, wc, sizeof(wc), cudaMemcpyHostToDevice, h->stream), "wall upload");
  OLB_CUDA(cudaStreamSynchronize(h->stream), "material sync");
  h->periodic = periodic_mask;
  h->has_bc = true;
  return OLB_OK;
}

int olb_ade_set_velocity_from(olb_ade_handle h, olb_handle fluid) {
  int rc = ade_check(h);
  if (rc) return rc;
  if ((rc = check(fluid))) return rc;
  if (fluid->nx != h->nx || fluid->ny != h->ny || fluid->nz != h->nz || fluid->dim != (h->q == 5 ? 2 : 3))
    return fail(OLB_ERR_ARG, "the fluid lattice does not match the advection-diffusion lattice");
  const size_t bytes = 3 * (size_t)h->ncell * sizeof(double);
  if ((rc = h->vfield.reserve(bytes))) return rc;
  // the fluid's state is final on its own stream; the moments run on this handle's
  cudaEvent_t ev;
  OLB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
  cudaError_t e = cudaEventRecord(ev, fluid->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, ev, 0);
  cudaEventDestroy(ev);
  OLB_CUDA(e, "stream order");
  HostParams p = fluid->params();
  p.stream = h->stream;
  OLB_CUDA(fluid->kt->moments(p, gather_of(fluid->repr), fluid->buf[fluid->cur].p, nullptr,
                              static_cast<double*>(h->vfield.p)),
           "fluid velocity");
  h->has_vfield = true;
  return OLB_OK;
}

int olb_ade_init(olb_ade_handle h, const double* C) {
  int rc = ade_check(h);
  if (rc) return rc;
  if (!C) return fail(OLB_ERR_ARG, "null scalar field");
  const void* dc = nullptr;
  if ((rc = ade_input(h, C, (size_t)h->ncell * sizeof(double), h->stage, &dc))) return rc;
  OLB_CUDA(ade_init(h->host(), static_cast<const double*>(dc), h->buf[h->cur].p), "advection-diffusion init");
  return OLB_OK;
}

int olb_ade_step(olb_ade_handle h, int64_t n) {
  int rc = ade_check(h);
  if (rc) return rc;
  if (n < 0) return fail(OLB_ERR_ARG, "negative step count");
  const AdeHost a = h->host();
  for (int64_t s = 0; s < n; ++s) {
    OLB_CUDA(ade_step(a, h->buf[h->cur].p, h->buf[1 - h->cur].p), "advection-diffusion step");
    h->cur = 1 - h->cur;
  }
  return OLB_OK;
}

int olb_ade_density(olb_ade_handle h, double* C) {
  int rc = ade_check(h);
  if (rc) return rc;
  if (!C) return fail(OLB_ERR_ARG, "null output");
  const size_t bytes = (size_t)h->ncell * sizeof(double);
  bool dev = false;
  if ((rc = locate(C, &dev, "density output"))) return rc;
  if (dev) {
    OLB_CUDA(ade_density(h->host(), h->buf[h->cur].p, C), "advection-diffusion density");
    return OLB_OK;
  }
  if ((rc = h->stage.reserve(bytes))) return rc;
  OLB_CUDA(ade_density(h->host(), h->buf[h->cur].p, static_cast<double*>(h->stage.p)), "advection-diffusion density");
  OLB_CUDA(cudaMemcpyAsync(C, h->stage.p, bytes, cudaMemcpyDeviceToHost, h->stream), "density copy");
  OLB_CUDA(cudaStreamSynchronize(h->stream), "density sync");
  return OLB_OK;
}

}  // extern "C"
