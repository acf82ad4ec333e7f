// olb_tma.cuh -- the pull step of the paired kernel with its populations staged in
// shared memory by the tensor memory accelerator (TMA).
//
// Why: the step streams 2 x q stored values per cell.  In k_step_pair every thread
// issues its 19 global loads itself, so the bytes in flight per SM are bounded by
// the resident warps and their registers, and the 16-bit instances, which need the
// most loads in flight per byte, run out of registers first (64 per thread at four
// blocks per SM, with spills).  Here one thread per block issues one bulk tensor
// copy per population for a whole tile of rows into shared memory, completing on an
// mbarrier; two or three tiles are in flight per block while the block's threads
// collide the previous one from shared memory.  The bytes in flight no longer
// depend on the warps, the loads need no per-thread address arithmetic, and the
// threads keep their registers for the collision.
//
// Tile: R rows of the full x extent of one z plane (R = 256 / (nx / 2), 512 cells;
// two x boxes when nx > 256).  For population i the copy takes rows y - c_iy of
// plane z - c_iz, so a thread finds f_i(x) = f*_i(x - c_i) at column x - c_ix of its
// own row (columns wrap in shared memory).  Rows that wrap across a periodic y face
// are copied one by one from the wrapped row; planes wrap across a periodic z face
// by their coordinate.  Everything after the loads -- domain-edge bounce-back from
// the cell's own global slots, the collision, own-slot and bounce-back stores, the
// statistics -- is pair_update of the paired kernel.
//
// Every wait on an mbarrier is bounded in time (kTmaWaitNs); a block that gives up
// records the failure in the handle's error word, waits (bounded again) for the
// copies it still has in flight, and returns.  The host reports the word as
// OLB_ERR_TIMEOUT.
#pragma once

#include <cuda.h>

namespace olb {

constexpr int kTmaMaxStages = 4;
constexpr unsigned long long kTmaWaitNs = 2000000000ull;  // default limit of one wait: 2 s
constexpr int kTmaBarrierBytes = 128;                        // barriers ahead of the tiles
constexpr int kTmaAlignSlack = 128;  // dynamic shared memory is aligned to 128 bytes inside the kernel

// Geometry of the tiled launch (host-computed).
struct TmaGeom {
  int rows;              // R: rows per tile
  int pairs;             // nx / 2: threads per row
  int nbx, bx;           // x boxes per row and their width (elements)
  int tiles_y;           // tiles per plane over the rows y0 .. y1
  int ntiles;            // tiles_y * (z1 - z0 + 1)
  int stages;            // tiles in flight per block (2 .. kTmaMaxStages)
  unsigned stage_bytes;  // bytes one tile brings (q boxes of R x nx elements)
  unsigned extra_tx;     // bytes expected beyond them: 0, except under failure injection (the waits then run out)
  unsigned box_slot;     // bytes between population slots of a stage (128-byte multiple)
  unsigned long long wait_ns;  // limit of one wait
  unsigned* err;         // error word of the handle (1: a wait timed out)
  int warp_issue;        // 1: the lanes of warp 0 issue one population's copies each; 0: thread 0 issues all
  int bulk1d;            // 1: plain bulk copies of contiguous row ranges instead of tensor-map boxes
  int release_early;     // 1: let the next grid launch when this one starts; 0: when its blocks finish
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of `bar` with the given parity, at most `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned long long limit_ns) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (global_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// One tiled copy of the 4-D population tensor (x, y, z, population) into shared
// memory, completing `bytes of the box` on `bar`.
__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y,
                                         int z, int q) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(q), "r"(smem_u32(bar))
      : "memory");
}

// One contiguous bulk copy (no tensor map) of `bytes` from global `src` into shared
// `dst`, completing on `bar`.  Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Issue the copies of tile t into stage s: by thread 0 alone (lane = -1: every
// population), or by the lanes of warp 0 (lane l issues population l; lane 0 also
// arms the barrier).
template <class L, class S, class PL>
__device__ __forceinline__ void tma_issue_tile(const Params<float>& p, const TmaGeom& g, const CUtensorMap* tmain,
                                               const CUtensorMap* trow, const PL& pl, unsigned char* data,
                                               unsigned long long* full, int t, int s, int lane) {
  const int zt = p.z0 + t / g.tiles_y;
  const int ya = p.y0 + (t % g.tiles_y) * g.rows;
  // the stage's previous contents were read through the generic proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane <= 0) mbar_expect_tx(&full[s], g.stage_bytes + g.extra_tx);
  const bool py = (p.periodic & 2u) != 0, pz = (p.periodic & 4u) != 0;
#pragma unroll
  for (int i = 0; i < L::Q; ++i) {
    if (lane >= 0 && lane != i) continue;
    unsigned char* dst = data + ((size_t)s * L::Q + i) * g.box_slot;
    int zs = zt - L::c(i, 2);
    if (pz) zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
    const int ys = ya - L::c(i, 1);
    if (g.bulk1d) {
      // rows outside a non-periodic face are taken from the nearest row: only edge
      // cells would read them, and those take such links from their own slots
      const int zc = zs < 0 ? 0 : (zs >= p.nz ? p.nz - 1 : zs);
      const size_t row_bytes = (size_t)p.nx * sizeof(S);
      if (ys >= 0 && ys + g.rows <= p.ny) {
        bulk_load(dst, pl.src[i] + ((size_t)zc * p.ny + ys) * p.nx, (unsigned)(g.rows * row_bytes), &full[s]);
      } else {
        for (int r = 0; r < g.rows; ++r) {
          int yr = ys + r;
          if (py)
            yr = yr < 0 ? yr + p.ny : (yr >= p.ny ? yr - p.ny : yr);
          else
            yr = yr < 0 ? 0 : (yr >= p.ny ? p.ny - 1 : yr);
          bulk_load(dst + r * row_bytes, pl.src[i] + ((size_t)zc * p.ny + yr) * p.nx, (unsigned)row_bytes, &full[s]);
        }
      }
      continue;
    }
    if (!py || (ys >= 0 && ys + g.rows <= p.ny)) {
      for (int b = 0; b < g.nbx; ++b)
        tma_load(dst + (size_t)b * g.bx * g.rows * sizeof(S), tmain, &full[s], b * g.bx, ys, zs, i);
    } else {
      for (int r = 0; r < g.rows; ++r) {
        int yr = ys + r;
        yr = yr < 0 ? yr + p.ny : (yr >= p.ny ? yr - p.ny : yr);
        for (int b = 0; b < g.nbx; ++b)
          tma_load(dst + ((size_t)r * p.nx + (size_t)b * g.bx) * sizeof(S), trow, &full[s], b * g.bx, yr, zs, i);
      }
    }
  }
}

// Loads from the staged tile with explicit shared-state-space instructions (a
// generic load would take the long path through the L1 pipeline).
template <class S>
struct SmemLoad;
template <>
struct SmemLoad<float> {
  __device__ static float ld1(unsigned a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
  }
  __device__ static F2 ld2(unsigned a) {
    float x, y;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(a));
    return F2(x, y);
  }
};
template <>
struct SmemLoad<__half> {
  __device__ static float ld1(unsigned a) {
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return __half2float(__ushort_as_half(v));
  }
  __device__ static F2 ld2(unsigned a) {
    unsigned v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
    __half2 h = *reinterpret_cast<__half2*>(&v);
    return F2(__half22float2(h));
  }
};
template <>
struct SmemLoad<__nv_bfloat16> {
  __device__ static float ld1(unsigned a) {
    unsigned short v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return __bfloat162float(__ushort_as_bfloat16(v));
  }
  __device__ static F2 ld2(unsigned a) {
    unsigned v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&v);
    return F2(__bfloat1622float2(h));
  }
};

// Pair of values of a population slot (shared address `slot`) at columns xa, xb of
// the row starting at element row_base.
template <class S>
__device__ __forceinline__ F2 sm_pair(unsigned slot, int row_base, int xa, int xb, bool adjacent) {
  if (adjacent) return SmemLoad<S>::ld2(slot + (unsigned)(row_base + xa) * sizeof(S));
  return F2(SmemLoad<S>::ld1(slot + (unsigned)(row_base + xa) * sizeof(S)),
            SmemLoad<S>::ld1(slot + (unsigned)(row_base + xb) * sizeof(S)));
}

template <class L, class S, bool STATS, bool WALLS, bool TRT>
__global__ void __launch_bounds__(256, 2)
    k_step_pair_tma(Params<float> p, const __grid_constant__ Planes<S, WALLS> pl,
                    const __grid_constant__ CUtensorMap tmain, const __grid_constant__ CUtensorMap trow, TmaGeom g,
                    double* partials) {
  // every copy lands at a 128-byte aligned shared address: the tile slots are
  // 128-byte multiples from a 128-byte aligned base
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem);
  unsigned char* data = smem + kTmaBarrierBytes;
  float sv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int tid = threadIdx.x;
  const int S_ = g.stages;
  if (tid == 0) {
    for (int s = 0; s < S_; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // bring both descriptors into the TMA unit's cache before the first copy
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&tmain)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&trow)) : "memory");
  }
  __syncthreads();
  // every block of this persistent grid is resident from the start: releasing the
  // next grid here would schedule it at once (see release_early); by default it is
  // released when each block has finished its tiles
  pdl_wait();
  if (g.release_early) pdl_release();
  // prologue: the first S - 1 tiles of this block
  const bool issuer = g.warp_issue ? tid < L::Q : tid == 0;
  const int lane = g.warp_issue ? tid : -1;
  if (issuer) {
    for (int j = 0; j + 1 < S_; ++j) {
      const int t = blockIdx.x + j * gridDim.x;
      if (t < g.ntiles) tma_issue_tile<L, S>(p, g, &tmain, &trow, pl, data, full, t, j, lane);
    }
  }
  const int r = tid / g.pairs;
  const int x0 = 2 * (tid - r * g.pairs);
  const bool lane_on = r < g.rows;
  int k = 0;
  for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x, ++k) {
    const int s = k % S_;
    const unsigned parity = (unsigned)(k / S_) & 1u;
    const int zt = p.z0 + t / g.tiles_y;
    const int y = p.y0 + (t % g.tiles_y) * g.rows + r;
    const bool on = lane_on && y <= p.y1;
    // the cell's link words and porosity do not come with the tile: load them
    // before waiting, so that their latency overlaps the wait
    const int cell = (zt * p.ny + (on ? y : p.y0)) * p.nx + x0;
    uint32_t w[2] = {kWordFluid, kWordFluid};
    if (WALLS && on) {
      const uint2 ww = *reinterpret_cast<const uint2*>(p.word + cell);
      w[0] = ww.x;
      w[1] = ww.y;
    }
    F2 gamma(1.0f);
    if (p.gamma && on) gamma = F2(*reinterpret_cast<const float2*>(p.gamma + cell));
    const bool ok = mbar_wait_bounded(&full[s], parity, g.wait_ns);
    if (__syncthreads_or(!ok)) {
      // give up: record it, let the copies still in flight (tiles k .. k + S - 2) land, return
      if (tid == 0) {
        atomicExch(g.err, 1u);
        for (int j = 0; j + 1 < S_; ++j) {
          const int kj = k + j;
          if (blockIdx.x + kj * gridDim.x < g.ntiles)
            mbar_wait_bounded(&full[kj % S_], (unsigned)(kj / S_) & 1u, g.wait_ns);
        }
      }
      __syncthreads();
      return;
    }
    // every thread is past tile k - 1: its stage takes tile k + S - 1
    if (issuer) {
      const int tn = t + (S_ - 1) * gridDim.x;
      if (tn < g.ntiles) tma_issue_tile<L, S>(p, g, &tmain, &trow, pl, data, full, tn, (k + S_ - 1) % S_, lane);
    }
    if (on) {
      const PairNbr n = make_pair_nbr<L>(p, x0, y, zt);
      const unsigned stage = smem_u32(data) + (unsigned)s * L::Q * g.box_slot;
      const int row_base = r * p.nx;
      F2 f[L::Q];
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const int cx = L::c(i, 0);
        f[i] = sm_pair<S>(stage + i * g.box_slot, row_base, n.xs[1 - cx], n.xs[2 - cx], cx == 0);
      }
      pair_update<L, S, G_PULL, S_OWN, STATS, WALLS, TRT>(p, pl, n, x0, y, zt, w, gamma, f, sv);
    }
  }
  if (!g.release_early) pdl_release();
  if (STATS) block_reduce_row(sv, partials + 8 * (int64_t)blockIdx.x, false);
}

}  // namespace olb
