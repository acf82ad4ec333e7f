// olb_oracle.cpp -- plain FP64 CPU oracle of the lattice Boltzmann BGK
// collide-and-stream map (OpenLB user guide, release 1.6, arXiv 2307.11752).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, literal reference that the
// GPU library is checked against.  Only the tests, the smoke check and the
// CPU-baseline leg of the benchmark load it.  It shares no code, header, table
// or constant with the CUDA library: the lattice tables below are typed in from
// the guide (D2Q9 listing, Descriptor section) and from the D3Q19 reading stated
// next to them.
//
// Every function follows the definition of the method written out loop by loop,
// in double precision, in the order of the guide's equations:
//   collision        f*_i = f_i + dt J_i,  J_i = -(f_i - f^eq_i)/tau   (section "Lattice
//                    Boltzmann Methods", collision and BGK equations; BGK listing in
//                    "Implementation in Dynamics": f <- (1-omega) f + omega f^eq)
//   streaming        f_i(t+1, x + c_i) = f*_i(t, x)                     (streaming equation)
//   moments          rho = sum_i f_i, rho u = sum_i c_i f_i             (moment summation, same section)
//   forcing          u_shift = u + F/2, Guo source term                 (Eqs. FBD and dF)
//   porosity         equilibrium velocity scaled by d in [0,1]          (section "Porous Media Model")
//   boundaries       BounceBack / BounceBackVelocity                    (section "Define Boundary Values")
// Points the guide leaves open are read as follows (the same readings are listed
// with their reasons in the design notes of the repository):
//   * equilibrium: textbook second-order truncation w rho (1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2)),
//     the second-order sibling of the first-order equilibrium printed in the
//     advection-diffusion section;
//   * bounce-back: link-wise halfway; a moving wall subtracts 2 w_i rho_x (c_i.u_w)/cs2,
//     rho_x the density of the fluid cell itself before collision;
//   * Guo forcing: u = (j + F/2)/rho (equal to the guide's u + F/2 at rho = 1) and the
//     source (1 - omega/2) w_i ((c_i - u)/cs2 + (c_i.u) c_i/cs2^2) . F with F a force density;
//   * porosity: the equilibrium and the Guo source use u' = gamma u; reported velocities
//     (moments, loss) use u;
//   * cells of material 0 (void), 2 (no-slip wall) and >= 3 (moving wall, velocity from the
//     wall table) are never collided; a link to such a cell, or out of the domain on a
//     non-periodic axis, bounces back (void and outside behave as no-slip walls);
//   * adjoint: the exact discrete adjoint (differentiate the discrete map), see the
//     reverse sweep below.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off [-fopenmp] -shared -fPIC.  The OpenMP
// pragmas only split independent cells over threads; every reduction is serial, so
// results do not depend on the thread count.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------------
// Lattice tables
// ---------------------------------------------------------------------------------
struct Desc {
  int d, q;
  int c[19][3];
  int opp[19];
  double w[19];
  double cs2;
};

// D2Q9 exactly as printed in the guide's listing "Definition of the D2Q9 descriptor"
// (section "Descriptor"): velocity order, opposite table, weights 4/9, 1/9, 1/36, cs2 = 1/3.
const Desc kD2Q9 = {
    2, 9,
    {{0, 0, 0}, {-1, 1, 0}, {-1, 0, 0}, {-1, -1, 0}, {0, -1, 0},
     {1, -1, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}},
    {0, 5, 6, 7, 8, 1, 2, 3, 4},
    {4.0 / 9.0, 1.0 / 36.0, 1.0 / 9.0, 1.0 / 36.0, 1.0 / 9.0,
     1.0 / 36.0, 1.0 / 9.0, 1.0 / 36.0, 1.0 / 9.0},
    1.0 / 3.0};

// D3Q19: the guide shows the set only as a figure (section "Lattice Boltzmann
// Methods").  Reading: rest + 6 face neighbours (weight 1/18) + 12 edge neighbours
// (weight 1/36), rest weight 1/3, cs2 = 1/3.  Ordering by the rule visible in the
// D2Q9 listing: 0 = rest, 1..9 = the velocities whose first non-zero component is
// -1, and i + 9 = -c_i, so opposite(i) = i +- 9.
const Desc kD3Q19 = {
    3, 19,
    {{0, 0, 0},
     {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {-1, -1, 0}, {-1, 1, 0},
     {-1, 0, -1}, {-1, 0, 1}, {0, -1, -1}, {0, -1, 1},
     {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, -1, 0},
     {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}},
    {0, 10, 11, 12, 13, 14, 15, 16, 17, 18, 1, 2, 3, 4, 5, 6, 7, 8, 9},
    {1.0 / 3.0,
     1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0,
     1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
     1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 36.0, 1.0 / 36.0,
     1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0},
    1.0 / 3.0};

const Desc* descriptor(int d) {
  if (d == 0) return &kD2Q9;
  if (d == 1) return &kD3Q19;
  return nullptr;
}

// ---------------------------------------------------------------------------------
// Forward-mode dual number (value + one directional derivative), the analogue of
// the guide's ADf<T,n> with n = 1 (section "Derivative Computation").
// ---------------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline double value(double a) { return a; }
inline double value(const Dual& a) { return a.v; }

}  // namespace

// ---------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------
extern "C" {

// Lattice description shared by every oracle call (all arrays caller-owned).
typedef struct {
  int32_t descriptor;      // 0 = D2Q9, 1 = D3Q19
  int32_t nx, ny, nz;      // nz = 1 for D2Q9
  uint32_t periodic;       // bit 0: x, bit 1: y, bit 2: z
  int32_t collision;       // 0 = BGK, 1 = TRT (two relaxation times, magic parameter below)
  const uint8_t* material; // nx*ny*nz, x fastest; 1 = fluid, 0 void, 2 wall, >= 3 moving wall
  const double* wall_u;    // [256][3] wall velocity per material number (rows 0..2 unused)
  double tau;              // BGK relaxation time, omega = 1/tau
  double force[3];         // uniform body force density F (Guo)
  const double* gamma;     // per-cell porosity in [0,1] or NULL (gamma = 1)
  double magic;            // TRT: Lambda = (1/omega+ - 1/2)(1/omega- - 1/2), omega+ = 1/tau
  const double* force_field;  // per-cell force density [3][n], or NULL (the uniform force above)
} olb_oracle_lattice;

// Objective of the adjoint, evaluated on the state after the last step.
//   kind 0: mean of u[component] over the fluid cells whose coordinate along
//           plane_axis equals plane_index (discrete plane mode of the flux functors,
//           section "Discrete Flux Functor");
//   kind 1: velocity misfit J = 1/2 sum over the fluid cells x of the region of
//           |u(x) - u*(x)|^2, the objective 1/2 int |u - u*|^2 dx of the guide's
//           optimisation examples (domainIdentification3d, testFlowOpti3d) with
//           dx = 1 in lattice units; u_target = u* as [3][cells], region = per cell
//           flag (nonzero: in the region; NULL: every fluid cell).  The sum runs over
//           the d components of the lattice.
typedef struct {
  int32_t plane_axis, plane_index, component;
  int32_t kind;
  const double* u_target;
  const uint8_t* region;
} olb_oracle_objective;

}  // extern "C"

namespace {

struct Geo {
  const Desc* D;
  int nx, ny, nz;
  int64_t n;
  unsigned periodic;
  const uint8_t* mat;
  explicit Geo(const olb_oracle_lattice* L)
      : D(descriptor(L->descriptor)), nx(L->nx), ny(L->ny), nz(L->nz),
        n((int64_t)L->nx * L->ny * L->nz), periodic(L->periodic), mat(L->material) {}
  int64_t index(int x, int y, int z) const { return ((int64_t)z * ny + y) * nx + x; }
  // Cell reached from (x,y,z) by adding (dx,dy,dz), wrapping periodic axes.
  // Returns -1 when the step leaves the domain along a non-periodic axis.
  int64_t neighbour(int x, int y, int z, int dx, int dy, int dz) const {
    int p[3] = {x + dx, y + dy, z + dz};
    int e[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
      if (p[a] < 0 || p[a] >= e[a]) {
        if (!(periodic & (1u << a))) return -1;
        p[a] = (p[a] % e[a] + e[a]) % e[a];
      }
    }
    return index(p[0], p[1], p[2]);
  }
  bool fluid(int64_t c) const { return c >= 0 && mat[c] == 1; }
};

bool valid(const olb_oracle_lattice* L) {
  if (!L || !descriptor(L->descriptor) || !L->material) return false;
  if (L->nx < 1 || L->ny < 1 || L->nz < 1) return false;
  if (L->descriptor == 0 && L->nz != 1) return false;
  if (!(L->tau > 0.5)) return false;
  if (L->collision != 0 && !(L->collision == 1 && L->magic > 0.0)) return false;
  return true;
}

// Second-order equilibrium (reading of equilibria::SecondOrder, see header).
template <class T>
void equilibrium(const Desc& D, T rho, const T u[3], T* feq) {
  T uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < D.q; ++i) {
    T cu = D.c[i][0] * u[0] + D.c[i][1] * u[1] + D.c[i][2] * u[2];
    feq[i] = D.w[i] * rho *
             (T(1.0) + cu / D.cs2 + cu * cu / (2.0 * D.cs2 * D.cs2) - uu / (2.0 * D.cs2));
  }
}

// Moments of one cell: rho = sum f, j = sum c f, u = (j + F/2)/rho.  F is a double
// or, for forward-mode derivatives with respect to the force, a T.
template <class T, class TF>
void moments(const Desc& D, const T* f, const TF F[3], T& rho, T j[3], T u[3]) {
  rho = T(0.0);
  j[0] = j[1] = j[2] = T(0.0);
  for (int i = 0; i < D.q; ++i) {
    rho += f[i];
    for (int a = 0; a < 3; ++a) j[a] += double(D.c[i][a]) * f[i];
  }
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * T(F[a])) / rho;
}

// One BGK collision of one cell with Guo forcing and porosity scaling.
//   f*_i = (1 - omega) f_i + omega f^eq_i(rho, gamma u) + (1 - omega/2) S_i(gamma u)
template <class T, class TF>
void collide_cell(const Desc& D, const T* f, T gamma, T omega, const TF Fin[3], T* fs) {
  const T F[3] = {T(Fin[0]), T(Fin[1]), T(Fin[2])};
  T rho, j[3], u[3];
  moments(D, f, F, rho, j, u);
  T up[3] = {gamma * u[0], gamma * u[1], gamma * u[2]};
  T feq[19];
  equilibrium(D, rho, up, feq);
  T uF = up[0] * F[0] + up[1] * F[1] + up[2] * F[2];
  for (int i = 0; i < D.q; ++i) {
    T cF = D.c[i][0] * F[0] + D.c[i][1] * F[1] + D.c[i][2] * F[2];
    T cu = D.c[i][0] * up[0] + D.c[i][1] * up[1] + D.c[i][2] * up[2];
    T S = D.w[i] * ((cF - uF) / D.cs2 + cu * cF / (D.cs2 * D.cs2));
    fs[i] = (T(1.0) - omega) * f[i] + omega * feq[i] + (T(1.0) - 0.5 * omega) * S;
  }
}

// One TRT collision (collision::TRT of the dynamics tuples, section "Dynamics"; the
// guide names the operator without printing it -- read as the two-relaxation-time
// operator of Ginzburg): with the even and odd parts g+-_i = (g_i +- g_opp(i))/2 of
// f, f^eq and the Guo source S,
//   f*_i = f_i - omega+ (f+_i - feq+_i) - omega- (f-_i - feq-_i)
//              + (1 - omega+/2) S+_i + (1 - omega-/2) S-_i,
// omega+ = 1/tau sets the viscosity, omega- follows from the magic parameter
// Lambda = (1/omega+ - 1/2)(1/omega- - 1/2).  omega- = omega+ is BGK.
template <class T, class TF>
void collide_cell_trt(const Desc& D, const T* f, T gamma, T omega_p, T omega_m, const TF Fin[3], T* fs) {
  const T F[3] = {T(Fin[0]), T(Fin[1]), T(Fin[2])};
  T rho, j[3], u[3];
  moments(D, f, F, rho, j, u);
  T up[3] = {gamma * u[0], gamma * u[1], gamma * u[2]};
  T feq[19], S[19];
  equilibrium(D, rho, up, feq);
  T uF = up[0] * F[0] + up[1] * F[1] + up[2] * F[2];
  for (int i = 0; i < D.q; ++i) {
    T cF = D.c[i][0] * F[0] + D.c[i][1] * F[1] + D.c[i][2] * F[2];
    T cu = D.c[i][0] * up[0] + D.c[i][1] * up[1] + D.c[i][2] * up[2];
    S[i] = D.w[i] * ((cF - uF) / D.cs2 + cu * cF / (D.cs2 * D.cs2));
  }
  for (int i = 0; i < D.q; ++i) {
    const int o = D.opp[i];
    T fp = T(0.5) * (f[i] + f[o]), fm = T(0.5) * (f[i] - f[o]);
    T ep = T(0.5) * (feq[i] + feq[o]), em = T(0.5) * (feq[i] - feq[o]);
    T sp = T(0.5) * (S[i] + S[o]), sm = T(0.5) * (S[i] - S[o]);
    fs[i] = f[i] - omega_p * (fp - ep) - omega_m * (fm - em) + (T(1.0) - T(0.5) * omega_p) * sp +
            (T(1.0) - T(0.5) * omega_m) * sm;
  }
}

// omega- of the TRT operator from omega+ and the magic parameter.
template <class T>
T omega_minus(T omega_p, double magic) {
  return T(1.0) / (T(magic) / (T(1.0) / omega_p - T(0.5)) + T(0.5));
}

// Force density at cell c: the T field Ff ([3][n], forward-mode runs), else the
// lattice's per-cell field, else its uniform force.
template <class T>
void cell_force(const olb_oracle_lattice* L, const T* Ff, int64_t n, int64_t c, T F[3]) {
  for (int a = 0; a < 3; ++a)
    F[a] = Ff ? Ff[a * n + c] : T(L->force_field ? L->force_field[a * n + c] : L->force[a]);
}

template <class T>
T gamma_at(const olb_oracle_lattice* L, const T* gamma, int64_t c) {
  if (gamma) return gamma[c];
  (void)L;
  return T(1.0);
}

// Collision of every fluid cell: fs = C(f); non-fluid cells copied unchanged.
template <class T>
void collide_field(const olb_oracle_lattice* L, const T* f, const T* gamma, T omega, T* fs,
                   const T* Ff = nullptr) {
  Geo g(L);
  const Desc& D = *g.D;
  const bool trt = L->collision == 1;
  const T om_m = trt ? omega_minus(omega, L->magic) : omega;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < g.n; ++c) {
    T fc[19], fsc[19];
    for (int i = 0; i < D.q; ++i) fc[i] = f[i * g.n + c];
    if (g.mat[c] == 1) {
      T F[3];
      cell_force(L, Ff, g.n, c, F);
      if (trt)
        collide_cell_trt(D, fc, gamma_at(L, gamma, c), omega, om_m, F, fsc);
      else
        collide_cell(D, fc, gamma_at(L, gamma, c), omega, F, fsc);
    } else {
      for (int i = 0; i < D.q; ++i) fsc[i] = fc[i];
    }
    for (int i = 0; i < D.q; ++i) fs[i * g.n + c] = fsc[i];
  }
}

// Streaming with boundaries (push form of the streaming equation):
//   for fluid x and every i: y = x + c_i;
//     y fluid      -> fout_i(y)     = fs_i(x)
//     y moving wall-> fout_opp(i)(x) = fs_i(x) - 2 w_i rho_x (c_i . u_w) / cs2
//     otherwise    -> fout_opp(i)(x) = fs_i(x)
// rho_x is the density of the pre-collision state fpre at x.  Non-fluid cells keep
// their values (copied from fs).
template <class T>
void stream_field(const olb_oracle_lattice* L, const T* fs, const T* fpre, T* fout) {
  Geo g(L);
  const Desc& D = *g.D;
  for (int64_t k = 0; k < (int64_t)D.q * g.n; ++k) fout[k] = fs[k];
#pragma omp parallel for schedule(static)
  for (int z = 0; z < g.nz; ++z) {
    for (int y = 0; y < g.ny; ++y) {
      for (int x = 0; x < g.nx; ++x) {
        int64_t c = g.index(x, y, z);
        if (g.mat[c] != 1) continue;
        T rho = T(0.0);
        for (int i = 0; i < D.q; ++i) rho += fpre[i * g.n + c];
        for (int i = 0; i < D.q; ++i) {
          int64_t t = g.neighbour(x, y, z, D.c[i][0], D.c[i][1], D.c[i][2]);
          if (g.fluid(t)) {
            fout[i * g.n + t] = fs[i * g.n + c];
          } else if (t >= 0 && g.mat[t] >= 3) {
            const double* uw = L->wall_u + 3 * g.mat[t];
            double cuw = D.c[i][0] * uw[0] + D.c[i][1] * uw[1] + D.c[i][2] * uw[2];
            fout[D.opp[i] * g.n + c] = fs[i * g.n + c] - 2.0 * D.w[i] * rho * cuw / D.cs2;
          } else {
            fout[D.opp[i] * g.n + c] = fs[i * g.n + c];
          }
        }
      }
    }
  }
}

template <class T>
void step_field(const olb_oracle_lattice* L, T* f, const T* gamma, T omega, int64_t nsteps,
                const T* Ff = nullptr) {
  Geo g(L);
  std::vector<T> fs((size_t)g.D->q * g.n), fo((size_t)g.D->q * g.n);
  for (int64_t s = 0; s < nsteps; ++s) {
    collide_field(L, f, gamma, omega, fs.data(), Ff);
    stream_field(L, fs.data(), f, fo.data());
    std::memcpy((void*)f, (const void*)fo.data(), sizeof(T) * fo.size());
  }
}

// Neumaier-compensated running sum (so the conservation pins are limited by the
// method, not by the summation).
struct Sum {
  double s = 0, c = 0;
  void add(double v) {
    double t = s + v;
    if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v; else c += (v - t) + s;
    s = t;
  }
  double get() const { return s + c; }
};

template <class T>
bool objective_cells(const Geo& g, const olb_oracle_objective* obj, std::vector<int64_t>& cells) {
  if (!obj) return false;
  if (obj->kind == 1) {
    if (!obj->u_target) return false;
    for (int64_t c = 0; c < g.n; ++c)
      if (g.mat[c] == 1 && (!obj->region || obj->region[c] != 0)) cells.push_back(c);
    return !cells.empty();
  }
  if (obj->kind != 0 || obj->plane_axis < 0 || obj->plane_axis > 2 || obj->component < 0 ||
      obj->component > 2)
    return false;
  int e[3] = {g.nx, g.ny, g.nz};
  if (obj->plane_index < 0 || obj->plane_index >= e[obj->plane_axis]) return false;
  for (int z = 0; z < g.nz; ++z)
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        int p[3] = {x, y, z};
        int64_t c = g.index(x, y, z);
        if (p[obj->plane_axis] == obj->plane_index && g.mat[c] == 1) cells.push_back(c);
      }
  return !cells.empty();
}

template <class T>
T loss_of(const olb_oracle_lattice* L, const T* f, const std::vector<int64_t>& cells,
          const olb_oracle_objective* obj, const T* Ff = nullptr) {
  Geo g(L);
  const Desc& D = *g.D;
  T acc = T(0.0);
  for (int64_t c : cells) {
    T fc[19], rho, j[3], u[3];
    for (int i = 0; i < D.q; ++i) fc[i] = f[i * g.n + c];
    T F[3];
    cell_force(L, Ff, g.n, c, F);
    moments(D, fc, F, rho, j, u);
    if (obj->kind == 1) {
      for (int a = 0; a < D.d; ++a) {
        T e = u[a] - T(obj->u_target[a * g.n + c]);
        acc += T(0.5) * e * e;
      }
    } else {
      acc += u[obj->component];
    }
  }
  return obj->kind == 1 ? acc : acc / double(cells.size());
}

// Jacobian of one collision, J[k][i] = d f*_k / d f_i, plus d f*/d gamma and
// d f*/d omega, written out from the collision formula by the chain rule through
// rho, u = (j + F/2)/rho and u' = gamma u.
//   BGK (trt = false): f*_k = f_k + omega (feq_k - f_k) + (1 - omega/2) S_k.
//   TRT (trt = true):  the even parts relax at omega, the odd parts at omega_m, and
//   omega_m depends on omega through the magic parameter (d omega_m / d omega =
//   domega_m), so d f*/d omega includes that chain.
//   dF[k][b] (optional) = d f*_k / d F_b of the cell's force density: through
//   u = (j + F/2)/rho (d u'_a / d F_b = gamma delta_ab / (2 rho)) and the explicit F of
//   the Guo source.
void collision_jacobian(const Desc& D, const double* f, double gamma, double omega,
                        const double F[3], double J[19][19], double dg[19], double dw[19],
                        bool trt = false, double omega_m = 0.0, double domega_m = 0.0,
                        double (*dF)[3] = nullptr) {
  double rho, j[3], u[3];
  moments(D, f, F, rho, j, u);
  double up[3] = {gamma * u[0], gamma * u[1], gamma * u[2]};
  double feq[19];
  equilibrium(D, rho, up, feq);
  double uF = up[0] * F[0] + up[1] * F[1] + up[2] * F[2];
  double cs2 = D.cs2;
  // d feq_k / d f_i, d S_k / d f_i, and their gamma derivatives; S_k itself; the
  // force derivatives of feq_k and S_k (EF, SF)
  double Ep[19][19], Sp[19][19], Eg[19], Sg[19], S[19], EF[19][3], SF[19][3];
  for (int k = 0; k < D.q; ++k) {
    double cu = D.c[k][0] * up[0] + D.c[k][1] * up[1] + D.c[k][2] * up[2];
    double cF = D.c[k][0] * F[0] + D.c[k][1] * F[1] + D.c[k][2] * F[2];
    // d feq_k / d rho (explicit) and d feq_k / d u'_a ; d S_k / d u'_a
    double dE_drho = feq[k] / rho;
    double dE_du[3], dS_du[3];
    for (int a = 0; a < 3; ++a) {
      dE_du[a] = D.w[k] * rho * (D.c[k][a] / cs2 + cu * D.c[k][a] / (cs2 * cs2) - up[a] / cs2);
      dS_du[a] = D.w[k] * (-F[a] / cs2 + D.c[k][a] * cF / (cs2 * cs2));
    }
    for (int i = 0; i < D.q; ++i) {
      double e = dE_drho, sd = 0.0;
      for (int a = 0; a < 3; ++a) {
        double du_df = gamma * (D.c[i][a] - u[a]) / rho;  // d u'_a / d f_i
        e += dE_du[a] * du_df;
        sd += dS_du[a] * du_df;
      }
      Ep[k][i] = e;
      Sp[k][i] = sd;
    }
    Eg[k] = dE_du[0] * u[0] + dE_du[1] * u[1] + dE_du[2] * u[2];
    Sg[k] = dS_du[0] * u[0] + dS_du[1] * u[1] + dS_du[2] * u[2];
    S[k] = D.w[k] * ((cF - uF) / cs2 + cu * cF / (cs2 * cs2));
    for (int b = 0; b < 3; ++b) {
      const double du = gamma / (2.0 * rho);  // d u'_b / d F_b
      EF[k][b] = dE_du[b] * du;
      SF[k][b] = dS_du[b] * du + D.w[k] * ((D.c[k][b] - up[b]) / cs2 + cu * D.c[k][b] / (cs2 * cs2));
    }
  }
  if (!trt) {
    for (int k = 0; k < D.q; ++k) {
      for (int i = 0; i < D.q; ++i)
        J[k][i] = (k == i ? 1.0 - omega : 0.0) + omega * Ep[k][i] + (1.0 - 0.5 * omega) * Sp[k][i];
      dg[k] = omega * Eg[k] + (1.0 - 0.5 * omega) * Sg[k];
      dw[k] = -f[k] + feq[k] - 0.5 * S[k];
      if (dF)
        for (int b = 0; b < 3; ++b) dF[k][b] = omega * EF[k][b] + (1.0 - 0.5 * omega) * SF[k][b];
    }
    return;
  }
  const double gp = 1.0 - 0.5 * omega, gm = 1.0 - 0.5 * omega_m;
  for (int k = 0; k < D.q; ++k) {
    const int o = D.opp[k];
    for (int i = 0; i < D.q; ++i) {
      // even and odd parts of the identity, of feq' and of S'
      double Ie = 0.5 * ((k == i ? 1.0 : 0.0) + (o == i ? 1.0 : 0.0));
      double Io = 0.5 * ((k == i ? 1.0 : 0.0) - (o == i ? 1.0 : 0.0));
      double Ee = 0.5 * (Ep[k][i] + Ep[o][i]), Eo = 0.5 * (Ep[k][i] - Ep[o][i]);
      double Se = 0.5 * (Sp[k][i] + Sp[o][i]), So = 0.5 * (Sp[k][i] - Sp[o][i]);
      J[k][i] = (k == i ? 1.0 : 0.0) - omega * (Ie - Ee) - omega_m * (Io - Eo) + gp * Se + gm * So;
    }
    dg[k] = omega * 0.5 * (Eg[k] + Eg[o]) + omega_m * 0.5 * (Eg[k] - Eg[o]) + gp * 0.5 * (Sg[k] + Sg[o]) +
            gm * 0.5 * (Sg[k] - Sg[o]);
    // d f*_k / d omega (even part) and d f*_k / d omega_m (odd part)
    double d_even = -(0.5 * (f[k] + f[o]) - 0.5 * (feq[k] + feq[o])) - 0.25 * (S[k] + S[o]);
    double d_odd = -(0.5 * (f[k] - f[o]) - 0.5 * (feq[k] - feq[o])) - 0.25 * (S[k] - S[o]);
    dw[k] = d_even + d_odd * domega_m;
    if (dF)
      for (int b = 0; b < 3; ++b)
        dF[k][b] = omega * 0.5 * (EF[k][b] + EF[o][b]) + omega_m * 0.5 * (EF[k][b] - EF[o][b]) +
                   gp * 0.5 * (SF[k][b] + SF[o][b]) + gm * 0.5 * (SF[k][b] - SF[o][b]);
  }
}

// Transpose of the streaming map (stationary and moving walls), applied to an
// adjoint field lam (q x n) of the post-streaming state:
//   lam*_i(x) = lam_i(x + c_i)        if x + c_i is fluid
//             = lam_opp(i)(x)         otherwise
// and the direct density dependence of the moving-wall term,
//   lam_direct(x) = sum over moving-wall links i of lam_opp(i)(x) * (-2 w_i c_i.u_w / cs2),
// which the caller adds to every population of x (d rho_x / d f_j = 1).
void stream_transpose(const olb_oracle_lattice* L, const double* lam, double* lams,
                      double* lam_direct) {
  Geo g(L);
  const Desc& D = *g.D;
  for (int64_t k = 0; k < (int64_t)D.q * g.n; ++k) lams[k] = 0.0;
  for (int64_t c = 0; c < g.n; ++c) lam_direct[c] = 0.0;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < g.nz; ++z)
    for (int y = 0; y < g.ny; ++y)
      for (int x = 0; x < g.nx; ++x) {
        int64_t c = g.index(x, y, z);
        if (g.mat[c] != 1) continue;
        double direct = 0.0;
        for (int i = 0; i < D.q; ++i) {
          int64_t t = g.neighbour(x, y, z, D.c[i][0], D.c[i][1], D.c[i][2]);
          if (g.fluid(t)) {
            lams[i * g.n + c] = lam[i * g.n + t];
          } else {
            lams[i * g.n + c] = lam[D.opp[i] * g.n + c];
            if (t >= 0 && g.mat[t] >= 3) {
              const double* uw = L->wall_u + 3 * g.mat[t];
              double cuw = D.c[i][0] * uw[0] + D.c[i][1] * uw[1] + D.c[i][2] * uw[2];
              direct += lam[D.opp[i] * g.n + c] * (-2.0 * D.w[i] * cuw / D.cs2);
            }
          }
        }
        lam_direct[c] = direct;
      }
}

// Transpose of the collision Jacobian at state f applied to lams (adjoint of the
// post-collision state); accumulates gradients with respect to gamma (per cell)
// and omega (scalar).
void collide_transpose(const olb_oracle_lattice* L, const double* f, const double* lams,
                       double* lam, double* dgamma, double* domega, double* dforce = nullptr) {
  Geo g(L);
  const Desc& D = *g.D;
  double omega = 1.0 / L->tau;
  // TRT: omega_m(omega) at fixed magic Lambda; with a = 1/omega - 1/2,
  // omega_m = 1/(Lambda/a + 1/2) and d omega_m / d omega = -omega_m^2 Lambda / (a^2 omega^2)
  const bool trt = L->collision == 1;
  const double omega_m = trt ? omega_minus(omega, L->magic) : omega;
  const double a = 1.0 / omega - 0.5;
  const double domega_m = trt ? -omega_m * omega_m * L->magic / (a * a * omega * omega) : 1.0;
  std::vector<double> dw_cell(g.n, 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < g.n; ++c) {
    if (g.mat[c] != 1) {
      for (int i = 0; i < D.q; ++i) lam[i * g.n + c] = 0.0;
      continue;
    }
    double fc[19], J[19][19], dg[19], dwk[19], dF[19][3], Fc[3];
    for (int i = 0; i < D.q; ++i) fc[i] = f[i * g.n + c];
    double gam = L->gamma ? L->gamma[c] : 1.0;
    cell_force<double>(L, nullptr, g.n, c, Fc);
    collision_jacobian(D, fc, gam, omega, Fc, J, dg, dwk, trt, omega_m, domega_m, dF);
    if (dforce)
      for (int b = 0; b < 3; ++b) {
        double v = 0.0;
        for (int k = 0; k < D.q; ++k) v += dF[k][b] * lams[k * g.n + c];
        dforce[b * g.n + c] += v;
      }
    double gsum = 0.0, wsum = 0.0;
    for (int i = 0; i < D.q; ++i) {
      double v = 0.0;
      for (int k = 0; k < D.q; ++k) v += J[k][i] * lams[k * g.n + c];
      lam[i * g.n + c] = v;
    }
    for (int k = 0; k < D.q; ++k) {
      gsum += dg[k] * lams[k * g.n + c];
      wsum += dwk[k] * lams[k * g.n + c];
    }
    if (dgamma) dgamma[c] += gsum;
    dw_cell[c] = wsum;
  }
  if (domega) {
    Sum s;
    for (int64_t c = 0; c < g.n; ++c) s.add(dw_cell[c]);
    *domega += s.get();
  }
}

// Force field as dual numbers: the lattice's force (value) with direction dir
// ([3][n]); an empty vector when dir is NULL (the plain double force is used).
std::vector<Dual> dual_force(const olb_oracle_lattice* L, int64_t n, const double* dir) {
  std::vector<Dual> Ff;
  if (!dir) return Ff;
  Ff.resize(3 * (size_t)n);
  for (int64_t c = 0; c < n; ++c) {
    double F[3];
    cell_force<double>(L, nullptr, n, c, F);
    for (int a = 0; a < 3; ++a) Ff[a * n + c] = Dual(F[a], dir[a * n + c]);
  }
  return Ff;
}

}  // namespace

extern "C" {

// Lattice tables for the pins: dim, q, c (q x 3), opposite (q), weights (q), cs2.
int olb_oracle_descriptor(int d, int* dim, int* q, int* c, int* opp, double* w, double* cs2) {
  const Desc* D = descriptor(d);
  if (!D) return -1;
  *dim = D->d;
  *q = D->q;
  for (int i = 0; i < D->q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = D->c[i][a];
    opp[i] = D->opp[i];
    w[i] = D->w[i];
  }
  *cs2 = D->cs2;
  return 0;
}

// Single-cell equilibrium f^eq(rho, u).
int olb_oracle_equilibrium(int d, double rho, const double* u, double* feq) {
  const Desc* D = descriptor(d);
  if (!D) return -1;
  double uu[3] = {u[0], u[1], u[2]};
  equilibrium(*D, rho, uu, feq);
  return 0;
}

// Single-cell collision (for brute-force pins).
int olb_oracle_collide_cell(int d, const double* f, double gamma, double tau,
                            const double* F, double* fs) {
  const Desc* D = descriptor(d);
  if (!D || !(tau > 0.5)) return -1;
  collide_cell(*D, f, gamma, 1.0 / tau, F, fs);
  return 0;
}

// Single-cell TRT collision with magic parameter Lambda.
int olb_oracle_collide_cell_trt(int d, const double* f, double gamma, double tau, double magic,
                                const double* F, double* fs) {
  const Desc* D = descriptor(d);
  if (!D || !(tau > 0.5) || !(magic > 0.0)) return -1;
  collide_cell_trt(*D, f, gamma, 1.0 / tau, omega_minus(1.0 / tau, magic), F, fs);
  return 0;
}

// f = f^eq(rho, u) on every cell (section "Define Initial Conditions", iniEquilibrium).
// rho: n, u: [3][n] (x, y, z components), f: [q][n].
int olb_oracle_init_equilibrium(const olb_oracle_lattice* L, const double* rho,
                                const double* u, double* f) {
  if (!valid(L)) return -1;
  Geo g(L);
  const Desc& D = *g.D;
  for (int64_t c = 0; c < g.n; ++c) {
    double uc[3] = {u[c], u[g.n + c], u[2 * g.n + c]};
    double feq[19];
    equilibrium(D, rho[c], uc, feq);
    for (int i = 0; i < D.q; ++i) f[i * g.n + c] = feq[i];
  }
  return 0;
}

// Post-collision field fs = C(f).
int olb_oracle_collide(const olb_oracle_lattice* L, const double* f, double* fs) {
  if (!valid(L)) return -1;
  collide_field<double>(L, f, L->gamma, 1.0 / L->tau, fs);
  return 0;
}

// Streamed field fout = S(fs; rho from fpre).
int olb_oracle_stream(const olb_oracle_lattice* L, const double* fs, const double* fpre,
                      double* fout) {
  if (!valid(L)) return -1;
  stream_field<double>(L, fs, fpre, fout);
  return 0;
}

// n full steps in place: f <- S(C(f)).
int olb_oracle_step(const olb_oracle_lattice* L, double* f, int64_t nsteps) {
  if (!valid(L) || nsteps < 0) return -1;
  step_field<double>(L, f, L->gamma, 1.0 / L->tau, nsteps);
  return 0;
}

// Per-cell rho (n) and u = (j + F/2)/rho ([3][n]); non-fluid cells get rho = u = 0.
int olb_oracle_moments(const olb_oracle_lattice* L, const double* f, double* rho, double* u) {
  if (!valid(L)) return -1;
  Geo g(L);
  const Desc& D = *g.D;
  for (int64_t c = 0; c < g.n; ++c) {
    if (g.mat[c] != 1) {
      rho[c] = 0.0;
      for (int a = 0; a < 3; ++a) u[a * g.n + c] = 0.0;
      continue;
    }
    double fc[19], r, j[3], uc[3];
    for (int i = 0; i < D.q; ++i) fc[i] = f[i * g.n + c];
    double Fc[3];
    cell_force<double>(L, nullptr, g.n, c, Fc);
    moments(D, fc, Fc, r, j, uc);
    rho[c] = r;
    for (int a = 0; a < 3; ++a) u[a * g.n + c] = uc[a];
  }
  return 0;
}

// Lattice statistics over fluid cells (lesson "Extract Data From a Simulation"):
// out = {sum rho, sum j_x, sum j_y, sum j_z (j = sum_i c_i f_i), sum |u|^2 / 2,
//        max |u|, number of cells with a non-finite population}.
int olb_oracle_diagnostics(const olb_oracle_lattice* L, const double* f, double* out) {
  if (!valid(L)) return -1;
  Geo g(L);
  const Desc& D = *g.D;
  Sum m, jx, jy, jz, e;
  double umax = 0.0, bad = 0.0;
  for (int64_t c = 0; c < g.n; ++c) {
    if (g.mat[c] != 1) continue;
    double fc[19], r, j[3], u[3];
    bool finite = true;
    for (int i = 0; i < D.q; ++i) {
      fc[i] = f[i * g.n + c];
      if (!std::isfinite(fc[i])) finite = false;
    }
    if (!finite) { bad += 1.0; continue; }
    double Fc[3];
    cell_force<double>(L, nullptr, g.n, c, Fc);
    moments(D, fc, Fc, r, j, u);
    m.add(r);
    jx.add(j[0]); jy.add(j[1]); jz.add(j[2]);
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    e.add(0.5 * uu);
    if (std::sqrt(uu) > umax) umax = std::sqrt(uu);
  }
  out[0] = m.get(); out[1] = jx.get(); out[2] = jy.get(); out[3] = jz.get();
  out[4] = e.get(); out[5] = umax; out[6] = bad;
  return 0;
}

// Objective value of state f.
int olb_oracle_loss(const olb_oracle_lattice* L, const double* f,
                    const olb_oracle_objective* obj, double* loss) {
  if (!valid(L)) return -1;
  Geo g(L);
  std::vector<int64_t> cells;
  if (!objective_cells<double>(g, obj, cells)) return -1;
  *loss = loss_of<double>(L, f, cells, obj);
  return 0;
}

// Tangent-linear (forward-mode) derivative of the objective after nsteps from f0
// in the direction (dgamma_dir per cell, dtau_dir): dloss = dL/dgamma . v + dL/dtau * s.
int olb_oracle_tangent(const olb_oracle_lattice* L, const double* f0, int64_t nsteps,
                       const olb_oracle_objective* obj, const double* dgamma_dir,
                       double dtau_dir, double* loss, double* dloss, const double* dforce_dir) {
  if (!valid(L) || nsteps < 0) return -1;
  Geo g(L);
  const Desc& D = *g.D;
  std::vector<int64_t> cells;
  if (!objective_cells<Dual>(g, obj, cells)) return -1;
  std::vector<Dual> f((size_t)D.q * g.n), gam(g.n);
  for (size_t k = 0; k < f.size(); ++k) f[k] = Dual(f0[k], 0.0);
  for (int64_t c = 0; c < g.n; ++c)
    gam[c] = Dual(L->gamma ? L->gamma[c] : 1.0, dgamma_dir ? dgamma_dir[c] : 0.0);
  // omega = 1/tau, d omega = -d tau / tau^2
  Dual omega = Dual(1.0, 0.0) / Dual(L->tau, dtau_dir);
  std::vector<Dual> Ff = dual_force(L, g.n, dforce_dir);
  const Dual* Fp = Ff.empty() ? nullptr : Ff.data();
  step_field<Dual>(L, f.data(), gam.data(), omega, nsteps, Fp);
  Dual Lv = loss_of<Dual>(L, f.data(), cells, obj, Fp);
  *loss = Lv.v;
  *dloss = Lv.d;
  return 0;
}

// Jacobian-vector products of the single sub-operators, for the transpose pins:
//   dfs = (dC/df) df + (dC/dgamma) dgamma + (dC/dtau) dtau   at state f
int olb_oracle_collide_tangent(const olb_oracle_lattice* L, const double* f, const double* df,
                               const double* dgamma, double dtau, double* dfs, const double* dforce) {
  if (!valid(L)) return -1;
  Geo g(L);
  const Desc& D = *g.D;
  std::vector<Dual> fd((size_t)D.q * g.n), fs((size_t)D.q * g.n), gam(g.n);
  for (size_t k = 0; k < fd.size(); ++k) fd[k] = Dual(f[k], df ? df[k] : 0.0);
  for (int64_t c = 0; c < g.n; ++c)
    gam[c] = Dual(L->gamma ? L->gamma[c] : 1.0, dgamma ? dgamma[c] : 0.0);
  Dual omega = Dual(1.0, 0.0) / Dual(L->tau, dtau);
  std::vector<Dual> Ff = dual_force(L, g.n, dforce);
  collide_field<Dual>(L, fd.data(), gam.data(), omega, fs.data(), Ff.empty() ? nullptr : Ff.data());
  for (size_t k = 0; k < fs.size(); ++k) dfs[k] = fs[k].d;
  return 0;
}

//   lam = (dC/df)^T lams;  dgamma += (dC/dgamma)^T lams;  dtau += (dC/dtau)^T lams
int olb_oracle_collide_adjoint(const olb_oracle_lattice* L, const double* f,
                               const double* lams, double* lam, double* dgamma, double* dtau,
                               double* dforce) {
  if (!valid(L)) return -1;
  double domega = 0.0;
  collide_transpose(L, f, lams, lam, dgamma, &domega, dforce);
  if (dtau) *dtau += -domega / (L->tau * L->tau);
  return 0;
}

//   lams = S^T lam (linear part), lam_direct = moving-wall density term per cell
int olb_oracle_stream_adjoint(const olb_oracle_lattice* L, const double* lam, double* lams,
                              double* lam_direct) {
  if (!valid(L)) return -1;
  stream_transpose(L, lam, lams, lam_direct);
  return 0;
}

// Discrete adjoint of "nsteps steps from f0, then the objective".  Keeps every
// forward state (the oracle runs on small lattices), then sweeps backwards:
//   lam^N            = dL/df^N
//   lam*^n           = S^T lam^{n+1}
//   lam^n            = (dC/df^n)^T lam*^n + moving-wall density term
//   dL/dgamma       += (dC/dgamma)^T lam*^n,   dL/domega += (dC/domega)^T lam*^n
//   dL/dtau          = -dL/domega / tau^2
// lambda0 (optional, q x n) receives dL/df^0.
int olb_oracle_adjoint(const olb_oracle_lattice* L, const double* f0, int64_t nsteps,
                       const olb_oracle_objective* obj, double* loss, double* dgamma,
                       double* dtau, double* lambda0, double* dforce) {
  if (!valid(L) || nsteps < 0) return -1;
  Geo g(L);
  const Desc& D = *g.D;
  std::vector<int64_t> cells;
  if (!objective_cells<double>(g, obj, cells)) return -1;
  size_t qn = (size_t)D.q * g.n;
  std::vector<std::vector<double>> states(nsteps + 1, std::vector<double>(qn));
  std::memcpy(states[0].data(), f0, sizeof(double) * qn);
  for (int64_t s = 0; s < nsteps; ++s) {
    states[s + 1] = states[s];
    step_field<double>(L, states[s + 1].data(), L->gamma, 1.0 / L->tau, 1);
  }
  const std::vector<double>& fN = states[nsteps];
  *loss = loss_of<double>(L, fN.data(), cells, obj);
  // Seed lam^N = dL/df^N, with d u_a / d f_i = (c_ia - u_a) / rho:
  //   plane mean of u_a:  (1/M) (c_ia - u_a) / rho
  //   velocity misfit:    sum_a (u_a - u*_a) (c_ia - u_a) / rho
  std::vector<double> lam(qn, 0.0), lams(qn), lamn(qn), direct(g.n);
  if (dforce)
    for (int64_t k = 0; k < 3 * g.n; ++k) dforce[k] = 0.0;
  for (int64_t c : cells) {
    double fc[19], r, j[3], u[3];
    for (int i = 0; i < D.q; ++i) fc[i] = fN[i * g.n + c];
    double Fc[3];
    cell_force<double>(L, nullptr, g.n, c, Fc);
    moments(D, fc, Fc, r, j, u);
    for (int i = 0; i < D.q; ++i) {
      double v = 0.0;
      if (obj->kind == 1) {
        for (int a = 0; a < D.d; ++a) v += (u[a] - obj->u_target[a * g.n + c]) * (D.c[i][a] - u[a]) / r;
      } else {
        const int a = obj->component;
        v = (D.c[i][a] - u[a]) / r / double(cells.size());
      }
      lam[i * g.n + c] = v;
    }
    // the objective's own dependence on the force, through u = (j + F/2)/rho
    if (dforce) {
      if (obj->kind == 1) {
        for (int a = 0; a < D.d; ++a) dforce[a * g.n + c] += (u[a] - obj->u_target[a * g.n + c]) / (2.0 * r);
      } else {
        dforce[obj->component * g.n + c] += 1.0 / (2.0 * r * double(cells.size()));
      }
    }
  }
  std::vector<double> gg(g.n, 0.0);
  double domega = 0.0;
  for (int64_t s = nsteps - 1; s >= 0; --s) {
    stream_transpose(L, lam.data(), lams.data(), direct.data());
    collide_transpose(L, states[s].data(), lams.data(), lamn.data(), gg.data(), &domega, dforce);
    for (int64_t c = 0; c < g.n; ++c) {
      if (g.mat[c] != 1) continue;
      for (int i = 0; i < D.q; ++i) lamn[i * g.n + c] += direct[c];
    }
    lam.swap(lamn);
  }
  if (dgamma) std::memcpy(dgamma, gg.data(), sizeof(double) * g.n);
  if (dtau) *dtau = -domega / (L->tau * L->tau);
  if (lambda0) std::memcpy(lambda0, lam.data(), sizeof(double) * qn);
  return 0;
}

}  // extern "C"

// =================================================================================
// Advection-diffusion (section "Advection--Diffusion Equation"): BGK on D2Q5 /
// D3Q7 for a passive scalar C transported by a prescribed velocity v,
//   g*_i = g_i - omega (g_i - g^eq_i),   g^eq_i = w_i C (1 + c_i . v / cs2),
//   C = sum_i g_i,  diffusivity mu = cs2 (tau - 1/2),
// followed by periodic streaming g_i(x + c_i, t + 1) = g*_i(x, t).  The guide
// prints the first-order equilibrium and names the D2Q5 / D3Q7 descriptors; their
// tables are read as: rest velocity first, then the face velocities in the D2Q9
// order (first non-zero component -1 first, opposite at i + (q-1)/2), weights
// fixed by sum w = 1 and sum w c_a c_b = cs2 delta_ab with the usual
// cs2 = 1/3 (D2Q5: w = 1/3, 1/6) and cs2 = 1/4 (D3Q7: w = 1/4, 1/8).
// =================================================================================
namespace {

struct AdeDesc {
  int d, q;
  int c[7][3];
  int opp[7];
  double w[7];
  double cs2;
};

const AdeDesc kD2Q5 = {
    2, 5,
    {{0, 0, 0}, {-1, 0, 0}, {0, -1, 0}, {1, 0, 0}, {0, 1, 0}},
    {0, 3, 4, 1, 2},
    {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0},
    1.0 / 3.0};

const AdeDesc kD3Q7 = {
    3, 7,
    {{0, 0, 0}, {-1, 0, 0}, {0, -1, 0}, {0, 0, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}},
    {0, 4, 5, 6, 1, 2, 3},
    {1.0 / 4.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0, 1.0 / 8.0},
    1.0 / 4.0};

const AdeDesc* ade_descriptor(int d) {
  if (d == 0) return &kD2Q5;
  if (d == 1) return &kD3Q7;
  return nullptr;
}

// v at cell c: per-cell field [3][n] or the uniform vector
inline void ade_velocity(const double* v, const double* vu, int64_t n, int64_t c, double out[3]) {
  for (int a = 0; a < 3; ++a) out[a] = v ? v[a * n + c] : (vu ? vu[a] : 0.0);
}

void ade_equilibrium(const AdeDesc& D, double C, const double v[3], double* geq) {
  for (int i = 0; i < D.q; ++i) {
    double cv = D.c[i][0] * v[0] + D.c[i][1] * v[1] + D.c[i][2] * v[2];
    geq[i] = D.w[i] * C * (1.0 + cv / D.cs2);
  }
}

bool ade_valid(const AdeDesc* D, int nx, int ny, int nz) {
  if (!D || nx < 1 || ny < 1 || nz < 1) return false;
  if (D->d == 2 && nz != 1) return false;
  return true;
}

}  // namespace

extern "C" {

int olb_oracle_ade_step_bc(int d, int nx, int ny, int nz, unsigned periodic, const uint8_t* material,
                           const double* wall_C, double tau, const double* v, const double* vu, double* g,
                           int64_t nsteps);

// Table of D2Q5 (d = 0) or D3Q7 (d = 1): dim, q, c[q][3], opposite[q], w[q], cs2.
int olb_oracle_ade_descriptor(int d, int* dim, int* q, int* c, int* opp, double* w, double* cs2) {
  const AdeDesc* D = ade_descriptor(d);
  if (!D) return -1;
  *dim = D->d;
  *q = D->q;
  for (int i = 0; i < D->q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = D->c[i][a];
    opp[i] = D->opp[i];
    w[i] = D->w[i];
  }
  *cs2 = D->cs2;
  return 0;
}

// g = g^eq(C, v) on every cell; C [n], v [3][n] or NULL with vu[3] uniform.
int olb_oracle_ade_init(int d, int nx, int ny, int nz, const double* C, const double* v,
                        const double* vu, double* g) {
  const AdeDesc* D = ade_descriptor(d);
  if (!ade_valid(D, nx, ny, nz) || !C || !g) return -1;
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t c = 0; c < n; ++c) {
    double vc[3], geq[7];
    ade_velocity(v, vu, n, c, vc);
    ade_equilibrium(*D, C[c], vc, geq);
    for (int i = 0; i < D->q; ++i) g[i * n + c] = geq[i];
  }
  return 0;
}

// nsteps BGK collide-and-stream steps on a fully periodic lattice, in place.
int olb_oracle_ade_step(int d, int nx, int ny, int nz, double tau, const double* v,
                        const double* vu, double* g, int64_t nsteps) {
  return olb_oracle_ade_step_bc(d, nx, ny, nz, 7u, nullptr, nullptr, tau, v, vu, g, nsteps);
}

// As olb_oracle_ade_step with boundaries.  material (cells, NULL = all 1):
//   1 = bulk cell (collided and streamed),
//   0 = no-flux wall: a link into it bounces back, g_opp(i)(x) = g*_i(x),
//   2..255 = Dirichlet cell of value wall_C[m] (the guide's constant-temperature
//       boundary, named without its scheme -- read as anti-bounce-back):
//       g_opp(i)(x) = -g*_i(x) + 2 w_i C_w, which fixes C_w at the link's midpoint.
// Links that leave the domain along a non-periodic axis (bit a of `periodic`
// clear) bounce back like a no-flux wall.  Non-bulk cells keep their values.
int olb_oracle_ade_step_bc(int d, int nx, int ny, int nz, unsigned periodic, const uint8_t* material,
                           const double* wall_C, double tau, const double* v, const double* vu, double* g,
                           int64_t nsteps) {
  const AdeDesc* D = ade_descriptor(d);
  if (!ade_valid(D, nx, ny, nz) || !(tau > 0.5) || !g || nsteps < 0) return -1;
  const int64_t n = (int64_t)nx * ny * nz;
  if (material && !wall_C)
    for (int64_t c = 0; c < n; ++c)
      if (material[c] >= 2) return -1;
  const double omega = 1.0 / tau;
  const int e[3] = {nx, ny, nz};
  std::vector<double> gs((size_t)D->q * n);
  for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < n; ++c) {
      if (material && material[c] != 1) {
        for (int i = 0; i < D->q; ++i) gs[i * n + c] = g[i * n + c];
        continue;
      }
      double C = 0.0;
      for (int i = 0; i < D->q; ++i) C += g[i * n + c];
      double vc[3], geq[7];
      ade_velocity(v, vu, n, c, vc);
      ade_equilibrium(*D, C, vc, geq);
      for (int i = 0; i < D->q; ++i) gs[i * n + c] = g[i * n + c] - omega * (g[i * n + c] - geq[i]);
    }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const int64_t c = ((int64_t)z * ny + y) * nx + x;
          if (material && material[c] != 1) continue;
          for (int i = 0; i < D->q; ++i) {
            int p[3] = {x + D->c[i][0], y + D->c[i][1], z + D->c[i][2]};
            bool inside = true;
            for (int a = 0; a < 3; ++a) {
              if (p[a] < 0 || p[a] >= e[a]) {
                if (periodic & (1u << a)) p[a] = (p[a] + e[a]) % e[a];
                else inside = false;
              }
            }
            const int64_t t = inside ? ((int64_t)p[2] * ny + p[1]) * nx + p[0] : -1;
            const int m = (t < 0) ? 0 : (material ? material[t] : 1);
            if (m == 1) {
              g[i * n + t] = gs[i * n + c];
            } else if (m >= 2) {
              g[D->opp[i] * n + c] = -gs[i * n + c] + 2.0 * D->w[i] * wall_C[m];
            } else {
              g[D->opp[i] * n + c] = gs[i * n + c];
            }
          }
        }
  }
  return 0;
}

// C = sum_i g_i per cell.
int olb_oracle_ade_density(int d, int nx, int ny, int nz, const double* g, double* C) {
  const AdeDesc* D = ade_descriptor(d);
  if (!ade_valid(D, nx, ny, nz) || !g || !C) return -1;
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t c = 0; c < n; ++c) {
    double s = 0.0;
    for (int i = 0; i < D->q; ++i) s += g[i * n + c];
    C[c] = s;
  }
  return 0;
}

}  // extern "C"
