/*
 * olb.h -- C ABI of the GB300 lattice Boltzmann library (libolb.so).
 *
 * The library advances the lattice Boltzmann BGK map of the OpenLB user guide
 * (release 1.6, arXiv 2307.11752) on one NVIDIA GPU:
 *   collision  f*_i = f_i - (f_i - f^eq_i)/tau          (section "Lattice Boltzmann Methods",
 *                                                        collision and BGK equations; BGK listing)
 *   streaming  f_i(t+1, x + c_i) = f*_i(t, x)           (streaming equation, same section)
 * on the D2Q9 lattice of the "Descriptor" listing and on D3Q19 (velocities and
 * ordering: rest, then (-1,0,0),(0,-1,0),(0,0,-1),(-1,-1,0),(-1,1,0),(-1,0,-1),
 * (-1,0,1),(0,-1,-1),(0,-1,1), then index i+9 = -c_i), with periodic axes,
 * halfway bounce-back walls and moving walls (BounceBack / BounceBackVelocity,
 * section "Define Boundary Values"), a uniform Guo body force (Eqs. FBD, dF) and
 * a per-cell porosity that scales the equilibrium velocity (section "Porous
 * Media Model").  olb_adjoint_run returns the gradient of a plane-averaged
 * velocity with respect to the porosity field and tau (the adjoint approach of
 * section "Derivative Computation", taken here as the exact discrete adjoint);
 * olb_adjoint_run_misfit does the same for the velocity misfit of the guide's
 * optimisation examples.  olb_set_trt selects the TRT collision instead of BGK
 * (forward and adjoint).  The olb_ade_* calls run a separate advection-diffusion
 * lattice (D2Q5 / D3Q7, section "Advection--Diffusion Equation").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Cells are numbered x fastest: cell = x + nx*(y + ny*z).  Population arrays
 *    are structure-of-arrays [q][cells] in the canonical, unshifted form:
 *    pre-collision populations f(t) in double precision.  Velocity arrays are
 *    [3][cells] (the z component is 0 on D2Q9).
 *  - Array arguments may point to device memory of the current device (or managed
 *    memory) or to host memory (pinned or pageable); the library asks the driver
 *    which one it is and stages host data through a device buffer.  Device memory
 *    of another GPU is refused with OLB_ERR_ARG.  The caller owns every array; the
 *    library only reads or writes it during the call (no pointer is kept).
 *  - A handle lives on the device that was current when it was created; every
 *    call on it except the destroy call needs that device current (OLB_ERR_ARG
 *    otherwise).
 *  - Work is queued on the handle's CUDA stream (olb_set_stream; default: the
 *    legacy default stream).  Calls that return data through host pointers
 *    synchronise that stream before returning; the others are asynchronous.
 *  - Every call returns an olb_status.  On failure nothing observable has changed
 *    in the handle and olb_last_error() describes the cause (thread-local string,
 *    valid until the next call on the same thread).
 *  - A handle is not thread-safe: one thread at a time per handle.
 */
#ifndef OLB_H
#define OLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct olb_lattice* olb_handle;

/* D2Q9 and D3Q19: the fluid lattices (olb_lattice_create).  D2Q5 and D3Q7: the
 * advection-diffusion lattices (olb_ade_create). */
typedef enum { OLB_D2Q9 = 0, OLB_D3Q19 = 1, OLB_D2Q5 = 2, OLB_D3Q7 = 3 } olb_descriptor;

/* Storage type of the populations on the GPU.  F64 and F32 store f_i - w_i and
 * compute in the same precision; the *_SHIFTED types store f_i - w_i in 16 bits
 * (round to nearest even) and compute in FP32. */
typedef enum {
  OLB_F64 = 0,
  OLB_F32 = 1,
  OLB_F16_SHIFTED = 2,
  OLB_BF16_SHIFTED = 3
} olb_dtype;

/* Propagation pattern: PULL keeps two population buffers and gathers each cell's
 * populations from its neighbours; AA keeps one buffer and alternates an
 * in-place local step with an in-place neighbour step.  Both compute the same map. */
typedef enum { OLB_PULL = 0, OLB_AA = 1 } olb_scheme;

typedef enum {
  OLB_OK = 0,
  OLB_ERR_ARG = -1,         /* invalid argument (null handle, bad size, tau <= 1/2, ...) */
  OLB_ERR_CUDA = -2,        /* a CUDA runtime call failed */
  OLB_ERR_OOM = -3,         /* the allocator returned no memory */
  OLB_ERR_STATE = -4,       /* call not valid in the handle's current state */
  OLB_ERR_NONFINITE = -5,   /* a NaN or Inf population was found */
  OLB_ERR_TIMEOUT = -6,     /* a kernel's bounded wait on its own asynchronous copies ran out (reported
                               by the next synchronising call; the state is then invalid) */
  OLB_ERR_UNSUPPORTED = -7  /* combination not implemented */
} olb_status;

/* Material numbers (section "Setting Material Numbers"). */
enum {
  OLB_MAT_VOID = 0,        /* outside the domain: acts as a no-slip wall, never updated */
  OLB_MAT_FLUID = 1,       /* collided and streamed */
  OLB_MAT_BOUNCE_BACK = 2  /* halfway no-slip wall */
  /* 3..255: moving walls, velocity set with olb_set_wall_velocity (default 0) */
};

/* Periodicity mask bits for olb_set_material. */
enum { OLB_PERIODIC_X = 1, OLB_PERIODIC_Y = 2, OLB_PERIODIC_Z = 4 };

/* Device-memory provider for every buffer a handle owns.  alloc(size, ctx) returns
 * device memory (at least 256-byte aligned) or NULL; free_(ptr, ctx) releases it.
 * Passing alloc == NULL restores cudaMalloc/cudaFree.  Process-wide; affects
 * buffers allocated after the call (each buffer is freed by the provider that
 * allocated it).  Returns OLB_OK. */
int olb_set_allocator(void* (*alloc)(size_t size, void* ctx),
                      void (*free_)(void* ptr, void* ctx), void* ctx);

/* Create a lattice of nx*ny*nz cells (nz must be 1 for D2Q9) on the current CUDA
 * device.  All cells start as fluid, no axis periodic, tau = 1, no force, no
 * porosity, populations at rest (f = w), scheme PULL, time 0.
 * Errors: OLB_ERR_ARG (sizes < 1, more than 2^31 - 1 cells, bad enum),
 *         OLB_ERR_OOM, OLB_ERR_CUDA. */
int olb_lattice_create(olb_descriptor d, int nx, int ny, int nz, olb_dtype t, olb_handle* out);

/* Release every buffer of the handle (after synchronising its stream). */
int olb_lattice_destroy(olb_handle h);

/* Stream for all later work of the handle (a cudaStream_t; NULL = legacy default). */
int olb_set_stream(olb_handle h, void* cuda_stream);

/* Switch the propagation pattern; the state is preserved. */
int olb_set_scheme(olb_handle h, olb_scheme s);

/* Material number of every cell (uint8 [cells]) and the periodic axes.  A link
 * from a fluid cell to a non-fluid cell, or out of the domain along a
 * non-periodic axis, is a halfway bounce-back link.  Populations of non-fluid
 * cells are undefined afterwards.  Errors: OLB_ERR_ARG (null array, mask > 7,
 * z periodic on D2Q9). */
int olb_set_material(olb_handle h, const uint8_t* material, unsigned periodic_mask);

/* Velocity u_w of moving-wall material `material_id` (3..255).  A population
 * reflected from such a wall gains 6 w_i rho_x (c_i . u_w), rho_x the density of
 * the fluid cell before collision (BounceBackVelocity). */
int olb_set_wall_velocity(olb_handle h, int material_id, const double u[3]);

/* BGK relaxation time (omega = 1/tau); selects the BGK collision.
 * Errors: OLB_ERR_ARG unless tau > 1/2. */
int olb_set_bgk(olb_handle h, double tau);

/* Selects the TRT collision (collision::TRT of the guide's dynamics tuples,
 * section "Dynamics", which names the operator without printing it; read as the
 * two-relaxation-time operator).  For each pair (i, opp(i)) the even part
 * (f_i + f_opp(i))/2 relaxes to the even part of f^eq at omega+ = 1/tau (which
 * sets the viscosity nu = (tau - 1/2)/3), the odd part at omega- given by the
 * magic parameter Lambda = (1/omega+ - 1/2)(1/omega- - 1/2); the Guo source is
 * split the same way.  Lambda = (tau - 1/2)^2 is BGK; Lambda = 3/16 puts halfway
 * bounce-back walls exactly at the wall for Poiseuille flow at every tau.
 * olb_set_bgk switches back.  olb_adjoint_run and olb_adjoint_run_misfit
 * differentiate the TRT map while it is selected; their dL/dtau holds the magic
 * parameter fixed (omega- follows tau).
 * Errors: OLB_ERR_ARG unless tau > 1/2 and magic > 0. */
int olb_set_trt(olb_handle h, double tau, double magic);

/* Uniform body force density F (Guo forcing with u = (j + F/2)/rho, Eqs. FBD, dF). */
int olb_set_force(olb_handle h, const double F[3]);

/* Per-cell force density F(x) (double [3][cells], host or device; the z row is
 * ignored on D2Q9): the external force field that the guide's descriptors carry
 * per cell (section "Lattice Boltzmann Methods": FORCE field; lesson on external
 * forces) and that testFlowOpti3d identifies.  While a field is set it replaces
 * the uniform force of olb_set_force in the collision (Guo forcing with the cell's
 * own F), in u = (j + F/2)/rho of olb_moments, olb_diagnostics and the objectives.
 * The values are copied (stored in the compute precision).  NULL removes the field.
 * Lattices with a field run the one-cell-per-thread step kernel. */
int olb_set_force_field(olb_handle h, const double* F);

/* Per-cell porosity gamma in [0,1] (double [cells]); the equilibrium and the
 * forcing term use gamma*u (section "Porous Media Model").  The values are
 * copied (stored in the compute precision).  NULL removes the field (gamma = 1).
 * Errors: OLB_ERR_ARG for values outside [0,1] or non-finite. */
int olb_set_porosity(olb_handle h, const double* gamma);

/* f = f^eq(rho, u) on every cell (section "Define Initial Conditions",
 * iniEquilibrium); rho: double [cells] or NULL (= 1); u: double [3][cells] or
 * NULL (= 0).  Resets the time counter to 0. */
int olb_init_equilibrium(olb_handle h, const double* rho, const double* u);

/* f += df on every fluid cell (df: double [q][cells]), e.g. a seeded perturbation. */
int olb_perturb_populations(olb_handle h, const double* df);

/* Replace / read the canonical state f(t) (double [q][cells], unshifted).
 * olb_get_populations writes non-fluid cells as 0. */
int olb_set_populations(olb_handle h, const double* f);
int olb_get_populations(olb_handle h, double* f);

/* Advance the state by n >= 0 collide-and-stream steps (asynchronous). */
int olb_step(olb_handle h, int64_t n);

/* Advance by n >= 1 steps like olb_step and return the lattice statistics that
 * the last step's collision evaluated (the state it collided, f(t + n - 1)), in
 * the layout of olb_diagnostics -- OpenLB's getStatistics() after a
 * collideAndStream ("evaluated during the previous collision step").  The
 * statistics are accumulated inside the fused step kernel; no extra pass over
 * the populations.  Synchronises the stream.  Returns OLB_ERR_NONFINITE (after
 * filling out) when a non-finite population was collided. */
int olb_step_stats(olb_handle h, int64_t n, double* out);

/* Density rho (double [cells]) and velocity u = (j + F/2)/rho (double [3][cells])
 * of the current state; non-fluid cells get 0.  Either pointer may be NULL. */
int olb_moments(olb_handle h, double* rho, double* u);

/* Lattice statistics of the current state over fluid cells (lesson "Extract
 * Data From a Simulation"), accumulated in double precision:
 *   out[0] sum rho, out[1..3] sum j (j = sum_i c_i f_i), out[4] sum |u|^2/2,
 *   out[5] max |u|, out[6] number of cells holding a NaN or Inf population
 * (such cells are left out of out[0..5]).  out is a host or device double[7];
 * returns OLB_ERR_NONFINITE (after filling out) when out[6] > 0. */
int olb_diagnostics(olb_handle h, double* out);

/* Objective of olb_adjoint_run: mean of u[component] over the fluid cells whose
 * coordinate along plane_axis (0 x, 1 y, 2 z) equals plane_index -- the discrete
 * plane reduction of the flux functors (section "Discrete Flux Functor"). */
typedef struct {
  int32_t plane_axis;
  int32_t plane_index;
  int32_t component;
} olb_objective;

/* Run n_steps steps from the current state, evaluate the objective L on the final
 * state, and return dL/dgamma (double [cells], 0 on non-fluid cells) and dL/dtau.
 * Forward states are checkpointed every `checkpoint_every` steps and each segment
 * is recomputed in reverse before its adjoint steps.  The handle ends in the final
 * forward state (time advanced by n_steps), as after olb_step(h, n_steps).
 * The gradient is with respect to the porosity field set by olb_set_porosity
 * (gamma = 1 everywhere when none is set).  Any of loss, dL_dgamma, dL_dtau may
 * be NULL.  Device memory: (ceil(n/K) + K) copies of the state plus two adjoint
 * fields (K = checkpoint_every).
 * Errors: OLB_ERR_ARG (n_steps < 1, K < 1, bad objective or empty plane),
 *         OLB_ERR_OOM. */
int olb_adjoint_run(olb_handle h, int64_t n_steps, int64_t checkpoint_every,
                    const olb_objective* obj, double* loss, double* dL_dgamma,
                    double* dL_dtau);

/* As olb_adjoint_run, for the velocity misfit
 *     J = 1/2 sum over the fluid cells x of the region of |u(x) - u*(x)|^2
 * on the final state: the objective 1/2 int |u - u*|^2 dx of the guide's
 * optimisation examples (section "optimization": domainIdentification3d, where a
 * porosity field is identified from a reference flow, and testFlowOpti3d), with
 * dx = 1 in lattice units.  u = (j + F/2)/rho as in olb_moments; the sum runs over
 * the lattice's d velocity components.
 *   u_target  double [3][cells] (layout of olb_moments' u; the z row is ignored for
 *             D2Q9), host or device memory, read during the call
 *   region    uint8 [cells], nonzero = in the region, host or device memory, or
 *             NULL (every fluid cell)
 * Outputs as olb_adjoint_run: loss = J, dL_dgamma = dJ/dgamma (double [cells],
 * device or host), dL_dtau = dJ/dtau.
 * Errors: OLB_ERR_ARG (n_steps < 1, K < 1, NULL u_target, region without fluid
 *         cells), OLB_ERR_OOM. */
int olb_adjoint_run_misfit(olb_handle h, int64_t n_steps, int64_t checkpoint_every,
                           const double* u_target, const uint8_t* region, double* loss,
                           double* dL_dgamma, double* dL_dtau);

/* Outputs of olb_adjoint_gradients; any pointer may be NULL (not computed).
 *   loss       host double: the objective
 *   dL_dgamma  double [cells], host or device: gradient with respect to the porosity
 *   dL_dtau    host double: gradient with respect to tau (TRT: magic parameter fixed)
 *   dL_dF      double [3][cells], host or device: gradient with respect to the force
 *              density of every cell (zero on non-fluid cells and, on D2Q9, in the z
 *              row), whether the force is a field or uniform: the control of the
 *              guide's force-field identification (testFlowOpti3d).  It collects the
 *              force's three routes: u = (j + F/2)/rho in the collision, the Guo
 *              source itself, and u in the objective. */
typedef struct {
  double* loss;
  double* dL_dgamma;
  double* dL_dtau;
  double* dL_dF;
} olb_gradients;

/* The checkpointed adjoint run of olb_adjoint_run (obj != NULL, u_target == NULL)
 * or of olb_adjoint_run_misfit (obj == NULL, u_target and region as there), with
 * every gradient output of olb_gradients.  dL_dF costs 3 double fields more device
 * memory and one read-modify-write of them per adjoint step.
 * Errors: as those calls; OLB_ERR_ARG also for out == NULL, or for both or neither
 *         of obj and u_target. */
int olb_adjoint_gradients(olb_handle h, int64_t n_steps, int64_t checkpoint_every, const olb_objective* obj,
                          const double* u_target, const uint8_t* region, olb_gradients* out);

/* Block the host until all work queued on the handle's stream has finished;
 * reports asynchronous CUDA errors as OLB_ERR_CUDA. */
int olb_synchronize(olb_handle h);

/* ---------------------------------------------------------------------------
 * Slab decomposition along z (the guide's parallel block decomposition with its
 * communicator, section "Communication": each block exchanges one layer of
 * populations with its neighbours per step).  A slab is an ordinary D3Q19 lattice
 * holding its share of the planes plus one halo plane on each z face: its material
 * carries the neighbouring slabs' planes there (void where the global lattice ends
 * on a non-periodic z face), and z is not periodic in it.  After each pull step the
 * populations leaving each interior face are packed, carried to the neighbouring
 * slab by any transport (a device copy between slabs on one GPU), and unpacked into
 * its halo plane; the next step then reads exactly what the single lattice would.
 * Only the pull scheme is supported.
 * --------------------------------------------------------------------------- */

/* Planes z_first .. z_last are updated by the steps and counted by olb_diagnostics;
 * the planes outside are halo planes.  (-1, -1) makes every plane active again.
 * Errors: OLB_ERR_ARG (empty or out-of-range). */
int olb_set_active_planes(olb_handle h, int z_first, int z_last);

/* Values per face buffer (populations crossing a z face times nx * ny) and the bytes
 * per value (the storage type's: buffers hold stored values unconverted). */
int olb_halo_size(olb_handle h, int64_t* values, int* elem_bytes);

/* Pack the populations that leave the active planes through face 0 (low z: those
 * with c_z = -1 at plane z_first) or face 1 (high z: c_z = +1 at plane z_last) into
 * buf, [population][y][x].  Unpack buf, packed by the neighbour across that face,
 * into the halo plane of face 0 (z_first - 1) or 1 (z_last + 1); only cells that
 * are fluid there receive values (a wall cell's slots hold its fluid neighbours'
 * bounce-back values).  buf is device memory of olb_halo_size values; queued on
 * the handle's stream.  Errors: OLB_ERR_STATE (no halo planes set, state not the one
 * after a pull step), OLB_ERR_UNSUPPORTED (not D3Q19), OLB_ERR_ARG. */
int olb_halo_pack(olb_handle h, int face, void* buf);
int olb_halo_unpack(olb_handle h, int face, const void* buf);

/* Failure injection for tests of the device-side timeout path (not for production
 * use; the guide has no counterpart).  The next step of the handle that runs the
 * TMA-fed pull kernel (FP32 or 16-bit storage, even nx, no force field; the state
 * after a pull step) expects `extra_bytes` more than its tile copies deliver, so
 * that the bounded wait of every block runs out after `wait_ns` nanoseconds.  The
 * blocks then record the failure, let their copies land and return: the step's
 * output is invalid, and the next synchronising call (olb_synchronize,
 * olb_step_stats, olb_diagnostics) returns OLB_ERR_TIMEOUT and clears it.  The
 * context stays usable.  Applies to one step; extra_bytes = 0 clears it.
 * Errors: OLB_ERR_ARG (extra_bytes > 65536, wait_ns outside [1e6, 5e9]). */
int olb_inject_stalled_copy(olb_handle h, unsigned extra_bytes, int64_t wait_ns);

/* Time step counter (steps since the last olb_init_equilibrium /
 * olb_set_populations) and the number of kernels the handle has launched. */
int olb_counters(olb_handle h, int64_t* time, int64_t* kernel_launches);

/* Lattice statistics (the 7 values of olb_diagnostics) of a canonical population
 * array, for callers that cannot allocate device memory: a process whose device
 * memory is already reserved by another allocator (such as a framework's caching
 * allocator), or a caller that cannot accept the device-wide synchronisation of
 * cudaMalloc/cudaFree.  This entry point allocates nothing: its per-block partial
 * sums live in a fixed array in the library's own device memory (4 MiB, held on
 * every GPU that loads the library until the process exits).  There is no
 * counterpart in the OpenLB guide; it is an interface of this library.
 *   f        device double [q][cells], canonical populations (as olb_get_populations)
 *   material device uint8 [cells] (1 = fluid; only fluid cells count) or NULL (all fluid)
 *   force    host double[3] used in u = (j + F/2)/rho, or NULL (no force)
 *   out      device double[7]: sum rho, sum j (3), sum |u|^2/2, max |u|, non-finite cells
 *   stream   cudaStream_t the work is queued on (asynchronous: out is ready when the
 *            stream reaches this point; non-finite cells are reported in out[6] only)
 * The first call on a device looks up the device address of the fixed array (with
 * that device current); make that first call before any stream capture.  All calls
 * on a device share the array, so calls that overlap on the GPU (on different
 * streams) race; order them on one stream.  Each call overwrites every partial sum
 * it reads, so no clearing is needed between calls.
 * The lookup is keyed on the device's current context, so after a device reset
 * the next call looks the address up again.
 * Errors: OLB_ERR_ARG for more than 16,777,216 cells (65,536 blocks of 256 cells,
 * the capacity of the fixed array), a bad descriptor or size, null f/out, or
 * arrays that are not device memory of the current device (host memory is not
 * staged: staging would allocate); OLB_ERR_CUDA for a failed launch. */
int olb_statistics_noalloc(olb_descriptor d, int nx, int ny, int nz, const double* f,
                           const uint8_t* material, const double* force, double* out,
                           void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Advection-diffusion of a passive scalar (section "Advection--Diffusion
 * Equation"): BGK on D2Q5 / D3Q7 towards the first-order equilibrium
 *     g^eq_i = w_i C (1 + c_i . v / cs2),   C = sum_i g_i,
 * diffusivity mu = cs2 (tau - 1/2); D2Q5: w = 1/3 (rest), 1/6, cs2 = 1/3; D3Q7:
 * w = 1/4, 1/8, cs2 = 1/4 (the guide names these descriptors without printing
 * their tables; the tables follow from sum w = 1 and sum w c_a c_b = cs2 delta).
 * Every axis is periodic unless olb_ade_set_material sets walls.  The velocity v is
 * prescribed (uniform or per cell) or taken from a fluid lattice.
 * The handle keeps the canonical state g(t) in two buffers of q x cells values
 * (F64 or F32), obtained through the olb_set_allocator provider.  Calls queue
 * work on the handle's stream (olb_ade_set_stream, default stream 0).
 * --------------------------------------------------------------------------- */
typedef struct olb_ade* olb_ade_handle;

/* descriptor OLB_D2Q5 (nz = 1) or OLB_D3Q7; dtype OLB_F64 or OLB_F32; tau = 1 and
 * v = 0 until set.  Errors: OLB_ERR_ARG, OLB_ERR_OOM. */
int olb_ade_create(int descriptor, int nx, int ny, int nz, int dtype, olb_ade_handle* out);
int olb_ade_destroy(olb_ade_handle h);
int olb_ade_set_stream(olb_ade_handle h, void* cuda_stream);
/* Relaxation time, tau > 1/2 (mu = cs2 (tau - 1/2)).  Errors: OLB_ERR_ARG. */
int olb_ade_set_tau(olb_ade_handle h, double tau);
/* Advection velocity: uniform v[3] (host), or per cell v_field double [3][cells]
 * (host or device, copied during the call; takes precedence when both are given).
 * The z component is ignored on D2Q5.  Errors: OLB_ERR_ARG (both NULL, non-finite). */
int olb_ade_set_velocity(olb_ade_handle h, const double v[3], const double* v_field);
/* Boundaries of the advection-diffusion lattice: material uint8 [cells] (host or
 * device) with 1 = bulk cell, 0 = no-flux wall (a link into it bounces back,
 * g_opp(i)(x) = g*_i(x)), 2..255 = Dirichlet cell of value wall_C[m] (the guide's
 * constant-temperature boundary, named without its scheme, read as anti-bounce-
 * back: g_opp(i)(x) = -g*_i(x) + 2 w_i C_w, which holds C_w at the link's midpoint);
 * periodic_mask: the axes that wrap (links leaving the domain along the others
 * bounce back like a no-flux wall); wall_C: double[256] on the host, or NULL when no
 * cell is Dirichlet.  Non-bulk cells keep their values.  Without this call every
 * cell is bulk and every axis periodic.
 * Errors: OLB_ERR_ARG (null material, bad mask, Dirichlet cells without wall_C,
 *         non-finite wall values). */
int olb_ade_set_material(olb_ade_handle h, const uint8_t* material, unsigned periodic_mask, const double* wall_C);

/* Advection velocity from a fluid lattice of the same size (D2Q9 for D2Q5, D3Q19
 * for D3Q7): v = u = (j + F/2)/rho of its current state, computed on the device
 * into this handle's velocity field (ordered after the fluid's queued work), so a
 * coupled step is olb_step(fluid, 1); olb_ade_set_velocity_from(h, fluid);
 * olb_ade_step(h, 1).  Errors: OLB_ERR_ARG (size or dimension mismatch). */
int olb_ade_set_velocity_from(olb_ade_handle h, olb_handle fluid);

/* g = g^eq(C, v) from C double [cells] (host or device). */
int olb_ade_init(olb_ade_handle h, const double* C);
/* n collide-and-stream steps. */
int olb_ade_step(olb_ade_handle h, int64_t n);
/* C = sum_i g_i into double [cells] (host: synchronises; device: queued). */
int olb_ade_density(olb_ade_handle h, double* C);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char* olb_last_error(void);

/* Static description of this build: target architecture and the compile-time
 * kernel configuration (for logs and benchmark records). */
const char* olb_build_info(void);

#ifdef __cplusplus
}
#endif

#endif /* OLB_H */
