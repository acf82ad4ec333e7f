// olb_pair.cuh -- step kernel that updates two neighbouring cells (x0, x0 + 1)
// per thread, for FP32 arithmetic (FP32, FP16 and BF16 storage).
//
// Why pairs: the update moves 2 x 19 stored values per cell against ~150 flops,
// and on sm_103a the FP32 arithmetic, the address arithmetic and the load/store
// instructions of one cell per thread fill the issue slots before the memory
// system is saturated.  Two cells per thread
//   * read and write the 9 populations with c_x = 0 as one 64-bit (FP32) or
//     32-bit (16-bit storage) access per pair, and every own-cell store likewise;
//   * run the collision in paired FP32 instructions (fma/add/mul .f32x2), one
//     instruction for both cells;
//   * share the neighbour-index arithmetic.
// Values stored in 16 bits are (f - w) * SCALE; the collision works directly in
// those units by writing the density as SCALE + delta_rho and the force as
// SCALE * F, so the scale costs no instruction.
#pragma once

// Included by olb_kernels.cuh after the shared definitions (Store, Params, Nbr,
// outside, on_edge, stats_of, block_reduce_row, lattice tables).

namespace olb {

// ---------------------------------------------------------------------------------
// Paired FP32 arithmetic.
// ---------------------------------------------------------------------------------
struct F2 {
  float2 v;
  __device__ F2() {}
  __device__ explicit F2(float s) : v(make_float2(s, s)) {}
  __device__ F2(float a, float b) : v(make_float2(a, b)) {}
  __device__ explicit F2(float2 a) : v(a) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return fma2(b, F2(-1.0f), a); }
__device__ __forceinline__ F2 neg(F2 a) { return a * F2(-1.0f); }

// Storage of populations in pairs.  SCALE: stored value = (f - w) * SCALE.
template <class S>
struct PairStore;
template <>
struct PairStore<float> {
  static constexpr float SCALE = 1.0f;
  static constexpr int MIN_BLOCKS = OLB_PAIR_MIN_BLOCKS;
  static constexpr int MIN_BLOCKS_WALLS = OLB_PAIR_MIN_BLOCKS;
  static constexpr int MIN_BLOCKS_TRT = OLB_PAIR_MIN_BLOCKS;
  static constexpr bool GHOST_FIRST = OLB_GHOST_FIRST32;
  static constexpr bool GHOST_COORDS = OLB_GHOST_COORDS32;
  __device__ static float ld1(const float* p) { return *p; }
  __device__ static F2 ld2(const float* p) { return F2(*reinterpret_cast<const float2*>(p)); }
  __device__ static void st1(float* p, float v) { *p = v; }
  __device__ static void st2(float* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }
};
template <>
struct PairStore<__half> {
  static constexpr float SCALE = Store<__half>::kScale;
  static constexpr int MIN_BLOCKS = OLB_PAIR16_MIN_BLOCKS;
  static constexpr int MIN_BLOCKS_WALLS = OLB_PAIR16_WALLS_MIN_BLOCKS;
  static constexpr int MIN_BLOCKS_TRT = OLB_PAIR16_TRT_MIN_BLOCKS;
  static constexpr bool GHOST_FIRST = OLB_GHOST_FIRST16;
  static constexpr bool GHOST_COORDS = OLB_GHOST_COORDS16;
  __device__ static float ld1(const __half* p) { return __half2float(*p); }
  __device__ static F2 ld2(const __half* p) { return F2(__half22float2(*reinterpret_cast<const __half2*>(p))); }
  __device__ static void st1(__half* p, float v) { *p = __float2half_rn(v); }
  __device__ static void st2(__half* p, F2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v); }
};
template <>
struct PairStore<__nv_bfloat16> {
  static constexpr float SCALE = 1.0f;
  static constexpr int MIN_BLOCKS = OLB_PAIR16_MIN_BLOCKS;
  static constexpr int MIN_BLOCKS_WALLS = OLB_PAIR16_WALLS_MIN_BLOCKS;
  static constexpr int MIN_BLOCKS_TRT = OLB_PAIR16_TRT_MIN_BLOCKS;
  static constexpr bool GHOST_FIRST = OLB_GHOST_FIRST16;
  static constexpr bool GHOST_COORDS = OLB_GHOST_COORDS16;
  __device__ static float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }
  __device__ static F2 ld2(const __nv_bfloat16* p) {
    return F2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p)));
  }
  __device__ static void st1(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ static void st2(__nv_bfloat16* p, F2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v.v);
  }
};

// Base pointers of the population planes of the source and destination buffers,
// passed as kernel parameters: each access is then one index add and one wide
// multiply-add on a constant-bank operand, instead of recomputing
// buffer + slot * pitch per access.
//
// The pointers' offset in the parameter space changes the generated code, and the
// instances differ in which offset they run faster with (measured at 128^3): the
// all-fluid FP32 step took 18% longer with its pointers at 8 mod 16 bytes than at
// 0 mod 16, while the instances with walls ran 1-3% faster at 8 mod 16.  So the
// struct is 16-byte aligned and LEAD = true puts one 8-byte word before the
// pointers; each instance takes its offset from that, not from sizeof(Params).
template <class S, bool LEAD>
struct alignas(16) Planes;
template <class S>
struct alignas(16) Planes<S, false> {
  const S* src[19];
  S* dst[19];
};
template <class S>
struct alignas(16) Planes<S, true> {
  unsigned long long lead;
  const S* src[19];
  S* dst[19];
};

// ---------------------------------------------------------------------------------
// Neighbourhood of a pair: x indices for offsets -1, 0, +1, +2 around x0 (wrapped)
// and the row bases of the 3 x 3 (dy, dz) offsets.
// ---------------------------------------------------------------------------------
struct PairNbr {
  int x0, y, z;
  int xs[4];  // x0 - 1, x0, x0 + 1, x0 + 2
  int row[3][3];
  __device__ __forceinline__ int at(int k, int dy, int dz) const { return row[dz + 1][dy + 1] + xs[k]; }
  __device__ __forceinline__ int cell() const { return row[1][1] + x0; }
};

template <class L>
__device__ __forceinline__ PairNbr make_pair_nbr(const Params<float>& p, int x0, int y, int z) {
  PairNbr n;
  n.x0 = x0;
  n.y = y;
  n.z = z;
  n.xs[0] = x0 == 0 ? p.nx - 1 : x0 - 1;
  n.xs[1] = x0;
  n.xs[2] = x0 + 1;
  n.xs[3] = x0 + 2 == p.nx ? 0 : x0 + 2;
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
  return n;
}

// Load the pair of values of slot `slot` at source cells (x0 + dx, x0 + 1 + dx) of
// the row offset (dy, dz): one paired access when dx == 0.
template <class S>
__device__ __forceinline__ F2 ld_pair(const S* plane, const PairNbr& n, int dx, int dy, int dz) {
  if (dx == 0) return PairStore<S>::ld2(plane + n.at(1, dy, dz));
  return F2(PairStore<S>::ld1(plane + n.at(1 + dx, dy, dz)), PairStore<S>::ld1(plane + n.at(2 + dx, dy, dz)));
}

template <class S>
__device__ __forceinline__ void st_pair(S* plane, const PairNbr& n, int dx, int dy, int dz, F2 v) {
  if (dx == 0) {
    PairStore<S>::st2(plane + n.at(1, dy, dz), v);
  } else {
    PairStore<S>::st1(plane + n.at(1 + dx, dy, dz), v.v.x);
    PairStore<S>::st1(plane + n.at(2 + dx, dy, dz), v.v.y);
  }
}

// BGK relaxation with omega w_k folded into the equilibrium's coefficients, per
// weight class (fewer instructions, a few more live registers).
#ifndef OLB_FOLD_OMEGA
#define OLB_FOLD_OMEGA 0
#endif

// ---------------------------------------------------------------------------------
// Collision of a pair in scaled units (values are (f - w) * SCALE).
//   rho_s = SCALE + sum f_s,  u = (j_s + F_s/2) / rho_s,  F_s = SCALE * F,
//   f*_s = f_s + omega (feq_s - f_s) + (1 - omega/2) Guo_s.
// Returns rho_s and u for the wall terms and statistics.
// ---------------------------------------------------------------------------------
// TRT = true: the two-relaxation-time operator (see collide in olb_kernels.cuh).
template <class L, int SCALE_NUM, bool TRT = false>
__device__ __forceinline__ void collide_pair(const Params<float>& p, F2 gamma, F2 (&f)[L::Q], F2& drho_s,
                                             F2 (&j_s)[3], F2& rho_s, F2 (&u)[3]) {
  constexpr float SCALE = (float)SCALE_NUM;
  // moments
  F2 d = f[0];
  F2 jj[3] = {F2(0.0f), F2(0.0f), F2(0.0f)};
#pragma unroll
  for (int k = 1; k <= L::HALF; ++k) {
    const int kp = k + L::HALF;
    d = d + f[k] + f[kp];
    const F2 a = f[kp] - f[k];
#pragma unroll
    for (int dd = 0; dd < 3; ++dd) {
      if (L::c(kp, dd) == 1) jj[dd] = jj[dd] + a;
      if (L::c(kp, dd) == -1) jj[dd] = jj[dd] - a;
    }
  }
  drho_s = d;
  j_s[0] = jj[0];
  j_s[1] = jj[1];
  j_s[2] = jj[2];
  const F2 rho = d + F2(SCALE);
  const F2 inv = F2(__frcp_rn(rho.v.x), __frcp_rn(rho.v.y));
  rho_s = rho;
  F2 up[3];
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    u[dd] = (jj[dd] + F2(p.half_force[dd] * SCALE)) * inv;
    up[dd] = gamma * u[dd];
  }
  F2 usq = up[0] * up[0];
  usq = fma2(up[1], up[1], usq);
  if (L::DIM == 3) usq = fma2(up[2], up[2], usq);
  const float om = p.omega;
  const F2 one_m_om(1.0f - om);
  const F2 omv(om);
  // A = drho_s - 1.5 rho_s usq ; B = 4.5 rho_s ; T = 3 rho_s
  const F2 A = fma2(F2(-1.5f) * rho, usq, d);
  const F2 B = F2(4.5f) * rho;
  const F2 T = F2(3.0f) * rho;
  const float gf = 1.0f - 0.5f * om;
  F2 uF(0.0f);
  if (p.forced) {
    uF = up[0] * F2(p.force[0] * SCALE);
    uF = fma2(up[1], F2(p.force[1] * SCALE), uF);
    uF = fma2(up[2], F2(p.force[2] * SCALE), uF);
  }
  {
    const float w0 = (float)L::w(0);
    F2 v = fma2(one_m_om, f[0], F2(om * w0) * A);
    if (p.forced) v = fma2(F2(-3.0f * gf * w0), uF, v);
    f[0] = v;
  }
#pragma unroll
  for (int k = 1; k <= L::HALF; ++k) {
    const int kp = k + L::HALF;
    const float wk = (float)L::w(k);
    F2 cu(0.0f);
    float cFs = 0.0f;
    bool first = true;
#pragma unroll
    for (int dd = 0; dd < L::DIM; ++dd) {
      const int c = L::c(kp, dd);
      if (c != 0) {
        if (first) {
          cu = c > 0 ? up[dd] : neg(up[dd]);
          first = false;
        } else {
          cu = c > 0 ? cu + up[dd] : cu - up[dd];
        }
        cFs += c * p.force[dd] * SCALE;
      }
    }
    F2 fp, fm;
    if (!TRT && OLB_FOLD_OMEGA) {
      // omega w_k (sym +- anti) with omega w_k folded into A, B and T once per weight
      // class (the products below are common to the directions of equal weight)
      const F2 symw = fma2(F2(om * wk * 4.5f) * rho, cu * cu, F2(om * wk) * A);
      const F2 antiw = F2(om * wk * 3.0f) * rho * cu;
      fp = fma2(one_m_om, f[kp], symw + antiw);
      fm = fma2(one_m_om, f[k], symw - antiw);
    } else if (!TRT) {
      const F2 sym = F2(wk) * fma2(B, cu * cu, A);
      const F2 anti = F2(wk) * T * cu;
      fp = fma2(one_m_om, f[kp], omv * (sym + anti));
      fm = fma2(one_m_om, f[k], omv * (sym - anti));
    } else {
      const F2 sym = F2(wk) * fma2(B, cu * cu, A);
      const F2 anti = F2(wk) * T * cu;
      // even = omega (f+ - sym), odd = omega_minus (f- - anti), f+- = (f_kp +- f_k)/2
      const F2 even = omv * fma2(F2(0.5f), f[kp] + f[k], neg(sym));
      const F2 odd = F2(p.omega_minus) * fma2(F2(0.5f), f[kp] - f[k], neg(anti));
      fp = f[kp] - (even + odd);
      fm = f[k] - (even - odd);
    }
    if (p.forced) {
      // Guo: gf w (9 cu cF - 3 u'.F) +- 3 gf w cF   (F in scaled units)
      const F2 gs = fma2(F2(9.0f * gf * wk * cFs), cu, F2(-3.0f * gf * wk) * uF);
      const float ga = 3.0f * (TRT ? 1.0f - 0.5f * p.omega_minus : gf) * wk * cFs;
      fp = fp + gs + F2(ga);
      fm = fm + gs - F2(ga);
    }
    f[kp] = fp;
    f[k] = fm;
  }
}

// 6 w_i (c_i . u_w) of wall material m (FP32 table).
template <class L>
__device__ __forceinline__ float wall_term_f(const Params<float>& p, int i, int m) {
  return p.wall_f[20 * m + i];
}

// Moving-wall part of the bounce-back of link i of a fluid cell with link word
// `word` (kWordMoving set): true and 6 w_i (c_i . u_w) in `t` when x + c_i is a
// moving wall.  The plane form of the word answers without a load; otherwise the
// neighbour's material is read.  tx indexes PairNbr::xs for x + c_i.
template <class L>
__device__ __forceinline__ bool moving_term(const Params<float>& p, int target, int i, uint32_t word, float& t) {
  const uint32_t code = (word >> kWordPlaneShift) & 7u;
  if (code) {
    const int a = (int)(code - 1) >> 1;
    const int s = (code & 1u) ? -1 : 1;
    const int ca = a == 0 ? L::c(i, 0) : (a == 1 ? L::c(i, 1) : L::c(i, 2));
    t = wall_term_f<L>(p, i, (int)((word >> kWordMatShift) & 255u));
    return ca == s;
  }
  const int wm = p.mat[target];
  if (wm < 3) return false;
  t = wall_term_f<L>(p, i, wm);
  return true;
}

// Index of the cell (x + dx, y + dy, z + dz), wrapped on every axis (a bounce-back
// link that crosses a lattice face crosses a periodic one: on the others the
// target is outside the lattice and the link is not a bounce-back link).  Built
// from the coordinates, so that the rare store paths that need it keep no
// neighbour indices live through the collision.
template <class L>
__device__ __forceinline__ int wrapped_cell(const Params<float>& p, int x, int y, int z, int dx, int dy, int dz) {
  int xt = x + dx, yt = y + dy, zt = z + dz;
  if (dx) xt = xt < 0 ? xt + p.nx : (xt >= p.nx ? xt - p.nx : xt);
  if (dy) yt = yt < 0 ? yt + p.ny : (yt >= p.ny ? yt - p.ny : yt);
  if (L::DIM == 3 && dz) zt = zt < 0 ? zt + p.nz : (zt >= p.nz ? zt - p.nz : zt);
  return (zt * p.ny + yt) * p.nx + xt;
}

// The push half step of the AA pattern stores to the neighbours: with 16-bit
// storage (64 registers) it rebuilds their indices from the coordinates after the
// collision rather than keeping them live across it.
#ifndef OLB_PUSH_RENBR16
#define OLB_PUSH_RENBR16 1
#endif
#ifndef OLB_PUSH_RENBR32
#define OLB_PUSH_RENBR32 0
#endif

// A copy of v that the compiler cannot prove equal to v and cannot compute before
// `after` (so that values derived from it are recomputed there, not kept live
// from before).
__device__ __forceinline__ int opaque(int v, float after) {
  asm volatile("" : "+r"(v) : "f"(after));
  return v;
}

// Special store paths for pairs at walls on the x faces (see the store phase).
#ifndef OLB_XWALL_PAIRS
#define OLB_XWALL_PAIRS 1
#endif
// Bounce-back stores of such pairs inside the own-slot loop (pull pattern).
#ifndef OLB_XWALL_GHOST16
#define OLB_XWALL_GHOST16 1
#endif
#ifndef OLB_XWALL_GHOST32
#define OLB_XWALL_GHOST32 1
#endif

// Link bits of the directions with c_x == cx (all non-rest directions for cx == 0
// is not used; see ghost_stores).
template <class L>
__host__ __device__ constexpr uint32_t dir_mask(int cx) {
  uint32_t m = 0;
  for (int i = 1; i < L::Q; ++i)
    if (L::c(i, 0) == cx) m |= 1u << i;
  return m;
}

// Bounce-back stores of cell h of a pair for the links set in `l`, testing only
// the directions with c_x == CX (CX == 0: all directions).
template <class L, class S, int SC, int CX, bool COORDS, class P>
__device__ __forceinline__ void ghost_stores(const Params<float>& p, const P& pl, const PairNbr& n, int h, int y,
                                             int z, uint32_t l, uint32_t word, float fh[L::Q], float rh) {
#pragma unroll
  for (int i = 1; i < L::Q; ++i) {
    if (CX != 0 && L::c(i, 0) != CX) continue;
    if (l & (1u << i)) {
      const int target = COORDS ? wrapped_cell<L>(p, n.x0 + h, y, z, L::c(i, 0), L::c(i, 1), L::c(i, 2))
                                : n.at(1 + h + L::c(i, 0), L::c(i, 1), L::c(i, 2));
      float v = fh[i];
      float t;
      if ((word & kWordMoving) && moving_term<L>(p, target, i, word, t)) v -= rh * t;  // rho_s 6 w c.u_w
      const int slot = (SC == S_OWN) ? opp<L>(i) : i;
      PairStore<S>::st1(pl.dst[slot] + target, v);
    }
  }
}

// ---------------------------------------------------------------------------------
// Everything after the population loads of one pair (x0, x0 + 1) of the step kernels:
// bounce-back at the domain edge (own-slot loads), collision, own-slot and
// bounce-back stores, statistics.  w: the cells' link words; f: f(t) of both cells
// (scaled shifted values); sv: the thread's statistics accumulators.
// ---------------------------------------------------------------------------------
template <class L, class S, int G, int SC, bool STATS, bool WALLS, bool TRT, class P>
__device__ __forceinline__ void pair_update(const Params<float>& p, const P& pl, const PairNbr& n, int x0, int y,
                                            int z, const uint32_t (&w)[2], F2 gamma, F2 (&f)[L::Q],
                                            float (&sv)[8]) {
  constexpr int SC_NUM = (int)PairStore<S>::SCALE;
  constexpr float INV_SCALE = 1.0f / PairStore<S>::SCALE;
  const int cell = n.cell();
  // links leaving the domain (no cell holds their bounce-back value)
  bool edge[2] = {false, false};
  if (WALLS && G != G_OWN && p.outside_links) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      Nbr c1;
      c1.x = x0 + h;
      c1.y = y;
      c1.z = z;
      edge[h] = on_edge<L>(p, x0 + h, y, z);
      if (edge[h]) {
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
          if (outside(p, c1, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2))) {
            const int own = (G == G_PULL) ? opp<L>(i) : i;
            const float v = PairStore<S>::ld1(pl.src[own] + cell + h);
            if (h == 0) f[i].v.x = v; else f[i].v.y = v;
          }
        }
      }
    }
  }
  F2 drho, j[3], rho, u[3];
  collide_pair<L, SC_NUM, TRT>(p, gamma, f, drho, j, rho, u);
  const bool fl0 = (w[0] & kWordFluid) != 0, fl1 = (w[1] & kWordFluid) != 0;
  if (!WALLS) {
    // every cell fluid, every axis periodic: plain paired stores only
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      if (SC == S_PUSH)
        st_pair(pl.dst[i], n, L::c(i, 0), L::c(i, 1), L::c(i, 2), f[i]);
      else
        PairStore<S>::st2(pl.dst[(SC == S_OWN) ? i : opp<L>(i)] + cell, f[i]);
    }
  } else if (SC == S_OWN || SC == S_OWN_SWAP) {
    // Own slots, one paired store per population.  A non-fluid cell's slots hold
    // nothing except its bounce-back slots (written by fluid neighbours, bits nb):
    // a pair whose non-fluid cell has bounce-back slots only on the side of its
    // fluid partner (the usual case at a wall on an x face) still stores in pairs,
    // except for the 5 directions that point from the non-fluid cell into its
    // partner, which store the fluid cell alone.
    const uint32_t nb0 = w[0] & kWordLinks, nb1 = w[1] & kWordLinks;
    const bool lo = OLB_XWALL_PAIRS && !fl0 && fl1 && !(nb0 & ~dir_mask<L>(1));   // non-fluid x0, fluid x0 + 1
    const bool hi = OLB_XWALL_PAIRS && fl0 && !fl1 && !(nb1 & ~dir_mask<L>(-1));  // fluid x0, non-fluid x0 + 1
    // Bounce-back links: the bounced population goes into the wall cell x + c_i,
    // in the slot that x reads there at the next step.  A cell next to a wall on
    // an x face has its links only among the 5 directions with c_x = -1 (or +1);
    // it tests only those.  These slots are never among the own slots stored
    // below (see above), so the bounce-back stores go first: the own-slot stores
    // then release the post-collision values one by one.
    //
    // In such a pair the fluid cell's links usually point at the x wall only.  Its
    // bounce-back targets are then the wall cells (x_wall, y + c_y, z + c_z), at a
    // fixed offset from its own index when y and z are not on a domain face (no
    // wrap-around).  Those stores go into the own-slot loop below as predicated
    // stores, so that the one boundary pair of a warp does not diverge from the
    // others; every other bounce-back link takes the per-cell path.
    bool interior = (unsigned)(y - 1) < (unsigned)(p.ny - 2);
    if (L::DIM == 3) interior = interior && (unsigned)(z - 1) < (unsigned)(p.nz - 2);
    constexpr bool XG = sizeof(S) == 2 ? OLB_XWALL_GHOST16 : OLB_XWALL_GHOST32;
    const bool lo_g = XG && lo && interior && !(nb1 & ~dir_mask<L>(-1)) && !(w[1] & kWordMoving);
    const bool hi_g = XG && hi && interior && !(nb0 & ~dir_mask<L>(1)) && !(w[0] & kWordMoving);
    const uint32_t l0 = (fl0 && !hi_g) ? nb0 : 0u;
    const uint32_t l1 = (fl1 && !lo_g) ? nb1 : 0u;
    auto bounce_back = [&]() {
    if (l0 | l1) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t l = h == 0 ? l0 : l1;
        if (l) {
          float fh[L::Q];
#pragma unroll
          for (int i = 0; i < L::Q; ++i) fh[i] = h == 0 ? f[i].v.x : f[i].v.y;
          const float rh = h == 0 ? rho.v.x : rho.v.y;
          if (OLB_XWALL_PAIRS && !(l & ~dir_mask<L>(-1)))
            ghost_stores<L, S, SC, -1, PairStore<S>::GHOST_COORDS>(p, pl, n, h, y, z, l, w[h], fh, rh);
          else if (OLB_XWALL_PAIRS && !(l & ~dir_mask<L>(1)))
            ghost_stores<L, S, SC, 1, PairStore<S>::GHOST_COORDS>(p, pl, n, h, y, z, l, w[h], fh, rh);
          else
            ghost_stores<L, S, SC, 0, PairStore<S>::GHOST_COORDS>(p, pl, n, h, y, z, l, w[h], fh, rh);
        }
      }
    }
    };
    if (PairStore<S>::GHOST_FIRST) bounce_back();
    if ((fl0 && fl1) || lo || hi) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        S* q = pl.dst[(SC == S_OWN) ? i : opp<L>(i)] + cell;
        if (L::c(i, 0) == 1 && lo) {
          PairStore<S>::st1(q + 1, f[i].v.y);
        } else if (L::c(i, 0) == -1 && hi) {
          PairStore<S>::st1(q, f[i].v.x);
        } else {
          PairStore<S>::st2(q, f[i]);
        }
        if (XG && L::c(i, 0) != 0) {
          // the x-wall bounce-back of this direction: cell x0 + 1 of a lo pair along
          // c_x = -1, cell x0 of a hi pair along c_x = +1, into slot opp(i) (S_OWN) of
          // the wall cell x + c_i
          const bool on = L::c(i, 0) == -1 ? (lo_g && ((nb1 >> i) & 1u)) : (hi_g && ((nb0 >> i) & 1u));
          if (on) {
            const int off = (L::c(i, 0) == -1 ? 0 : 1) + L::c(i, 1) * p.nx + (L::DIM == 3 ? L::c(i, 2) * p.nx * p.ny : 0);
            PairStore<S>::st1(pl.dst[(SC == S_OWN) ? opp<L>(i) : i] + cell + off,
                              L::c(i, 0) == -1 ? f[i].v.y : f[i].v.x);
          }
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        S* q = pl.dst[(SC == S_OWN) ? i : opp<L>(i)] + cell;
        if (fl0) PairStore<S>::st1(q, f[i].v.x);
        if (fl1) PairStore<S>::st1(q + 1, f[i].v.y);
      }
    }
    if (!PairStore<S>::GHOST_FIRST) bounce_back();
    if (OLB_SOLID_FILL) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!(h == 0 ? fl0 : fl1)) {
          const uint32_t nb = w[h] & kWordLinks;
#pragma unroll
          for (int k = 0; k < L::Q; ++k) {
            const int b = (SC == S_OWN) ? k : opp<L>(k);
            if (k == 0 || !(nb & (1u << b))) PairStore<S>::st1(pl.dst[k] + cell + h, 0.0f);
          }
        }
      }
    }
  } else {  // S_PUSH
    constexpr bool RENBR = sizeof(S) == 2 ? OLB_PUSH_RENBR16 : OLB_PUSH_RENBR32;
    const PairNbr m = RENBR ? make_pair_nbr<L>(p, opaque(x0, f[0].v.x), opaque(y, f[0].v.x), opaque(z, f[0].v.x)) : n;
    const uint32_t lk0 = w[0] & (kWordLinks | kWordMoving), lk1 = w[1] & (kWordLinks | kWordMoving);
    const bool plain = fl0 && fl1 && !(lk0 | lk1) && !edge[0] && !edge[1];
    // A pair at a wall on an x face: one cell non-fluid with fluid neighbours only on
    // its partner's side, the fluid cell with wall links only in the directions that
    // point at the wall's side (no moving wall, no domain edge).  In this half step
    // every slot is read and written by one cell only.  The non-fluid cell's values may
    // then go with its partner's paired stores in the directions with c_x = 0: the
    // slots they reach are non-fluid cells' and read by the non-fluid cell alone.  Not
    // along c_x = +-1, where they could hit a fluid cell's own bounce-back slot.  The
    // fluid cell's wall links store in its own slots.  Such pairs take the plain store
    // sequence with predicated stores and selected addresses, so a warp holding one
    // does not diverge.
    const uint32_t nb0 = w[0] & kWordLinks, nb1 = w[1] & kWordLinks;  // non-fluid cells: fluid neighbours
    const bool lo = OLB_XWALL_PAIRS && !fl0 && fl1 && !(nb0 & ~dir_mask<L>(1)) && !(lk1 & ~dir_mask<L>(-1)) &&
                    !edge[1];
    const bool hi = OLB_XWALL_PAIRS && fl0 && !fl1 && !(nb1 & ~dir_mask<L>(-1)) && !(lk0 & ~dir_mask<L>(1)) &&
                    !edge[0];
    if (plain || lo || hi) {
#pragma unroll
      for (int i = 0; i < L::Q; ++i) {
        const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        if (cx == 0) {
          st_pair(pl.dst[i], m, 0, cy, cz, f[i]);
        } else if (cx == 1) {
          // cell x0 streams to x0 + 1 (or, in a hi pair, bounces into its own slot);
          // cell x0 + 1 streams to x0 + 2 (not in a hi pair: it is the wall)
          S* a = (hi && ((lk0 >> i) & 1u)) ? pl.dst[opp<L>(i)] + cell : pl.dst[i] + m.at(2, cy, cz);
          if (!lo) PairStore<S>::st1(a, f[i].v.x);
          if (!hi) PairStore<S>::st1(pl.dst[i] + m.at(3, cy, cz), f[i].v.y);
        } else {
          // cell x0 streams to x0 - 1 (not in a lo pair); cell x0 + 1 streams to x0 (or,
          // in a lo pair, bounces into its own slot)
          if (!lo) PairStore<S>::st1(pl.dst[i] + m.at(0, cy, cz), f[i].v.x);
          S* b = (lo && ((lk1 >> i) & 1u)) ? pl.dst[opp<L>(i)] + cell + 1 : pl.dst[i] + m.at(1, cy, cz);
          if (!hi) PairStore<S>::st1(b, f[i].v.y);
        }
      }
    } else {
      // per cell, with bounce-back links, domain edges and non-fluid cells
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t wd = w[h];
        const int c = cell + h;
        const float rh = h == 0 ? rho.v.x : rho.v.y;
        Nbr c1;
        c1.x = x0 + h;
        c1.y = y;
        c1.z = z;
        if (wd & kWordFluid) {
#pragma unroll
          for (int i = 0; i < L::Q; ++i) {
            const float fi = h == 0 ? f[i].v.x : f[i].v.y;
            const int tx = 1 + h + L::c(i, 0);
            const bool wall = i != 0 && (wd & (1u << i));
            const bool out = i != 0 && edge[h] && outside(p, c1, L::c(i, 0), L::c(i, 1), L::c(i, 2));
            if (wall || out) {
              float bounced = fi;
              float t;
              if (wall && (wd & kWordMoving) &&
                  moving_term<L>(p, m.at(tx, L::c(i, 1), L::c(i, 2)), i, wd, t))
                bounced -= rh * t;
              PairStore<S>::st1(pl.dst[opp<L>(i)] + c, bounced);
            } else {
              PairStore<S>::st1(pl.dst[i] + m.at(tx, L::c(i, 1), L::c(i, 2)), fi);
            }
          }
        } else if (OLB_SOLID_FILL) {
          const uint32_t nb = wd & kWordLinks;
#pragma unroll
          for (int k = 0; k < L::Q; ++k)
            if (k == 0 || !(nb & (1u << opp<L>(k)))) PairStore<S>::st1(pl.dst[k] + c, 0.0f);
        }
      }
    }
  }
  if (STATS) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (w[h] & kWordFluid) {
        const float dr = (h == 0 ? drho.v.x : drho.v.y) * INV_SCALE;
        float jv[3], uv[3], v[8];
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) {
          jv[dd] = (h == 0 ? j[dd].v.x : j[dd].v.y) * INV_SCALE;
          uv[dd] = h == 0 ? u[dd].v.x : u[dd].v.y;
        }
        stats_of(dr, jv, uv, v);
#pragma unroll
        for (int k = 0; k < 8; ++k) sv[k] = (k == 5) ? fmaxf(sv[k], v[k]) : sv[k] + v[k];
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// The paired step kernel (patterns as in k_step, see scatter for the bounce-back
// storage rules).  Requires nx even; tiles of (2 << tile_shift) cells along x by
// (256 >> tile_shift) rows.  WALLS = false is the instance for lattices whose cells
// are all fluid with every axis periodic: it carries no boundary code at all, so
// the boundary paths cannot cost registers or scheduling freedom there.
// ---------------------------------------------------------------------------------
template <class L, class S, int G, int SC, bool STATS, bool WALLS, bool TRT>
__global__ void __launch_bounds__(256, TRT ? PairStore<S>::MIN_BLOCKS_TRT
                                            : (WALLS ? PairStore<S>::MIN_BLOCKS_WALLS : PairStore<S>::MIN_BLOCKS))
    k_step_pair(Params<float> p, const __grid_constant__ Planes<S, WALLS> pl, double* partials) {
  float sv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int tid = threadIdx.x;
  pdl_wait_then_release();
  int x0, y, z;
  bool active;
  {
    z = p.z0 + blockIdx.z;
    x0 = 2 * ((blockIdx.x << p.tile_shift) + (tid & ((1 << p.tile_shift) - 1)));
    y = p.y0 + blockIdx.y * (256 >> p.tile_shift) + (tid >> p.tile_shift);
    active = x0 < p.nx && y <= p.y1;
  }
  if (active) {
    const PairNbr n = make_pair_nbr<L>(p, x0, y, z);
    const int cell = n.cell();
    uint32_t w[2] = {kWordFluid, kWordFluid};
    if (WALLS) {
      const uint2 ww = *reinterpret_cast<const uint2*>(p.word + cell);
      w[0] = ww.x;
      w[1] = ww.y;
    }
    F2 f[L::Q];
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
      const int slot = (G == G_OWN || G == G_PULL) ? i : opp<L>(i);
      if (G == G_OWN)
        f[i] = PairStore<S>::ld2(pl.src[i] + cell);
      else
        f[i] = ld_pair(pl.src[slot], n, -L::c(i, 0), -L::c(i, 1), -L::c(i, 2));
    }
    F2 gamma(1.0f);
    if (p.gamma) gamma = F2(*reinterpret_cast<const float2*>(p.gamma + cell));
    pair_update<L, S, G, SC, STATS, WALLS, TRT>(p, pl, n, x0, y, z, w, gamma, f, sv);
  }
  if (STATS) block_reduce_row(sv, partials + 8 * block_linear(), false);
}

}  // namespace olb
