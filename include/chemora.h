/*
 * chemora.h -- C ABI of the GB300 (sm_103a) FP64 finite-difference + RK4 hot
 * path of the Chemora method (Schnetter et al., "Chemora: A PDE Solving
 * Framework for Modern HPC Architectures", arXiv 1410.1764).
 *
 * The paper describes the problem these calls solve: evaluate the right-hand
 * side (RHS) of a system of time-dependent PDEs with finite-difference
 * stencils on a uniform Cartesian grid with ghost zones (Sec. 2, driver and
 * ghost zones; Sec. 3.2.2, discretisation), and advance it with a Runge-Kutta
 * method of lines (Sec. 2, time integrator).  Systems: the scalar wave
 * equation (Sec. 3, Eq. 1), a variable-speed wave equation, and the Einstein
 * equations in BSSN form (Sec. 3.4, Sec. 5).
 *
 * Conventions (every entry point):
 *  - All `double*` arguments are DEVICE pointers owned by the caller unless
 *    stated otherwise.  Handles and their scratch memory are owned by the
 *    library and released by chemora_destroy.
 *  - A grid function is a contiguous FP64 array [nz+2g][ny+2g][nx+2g], x
 *    fastest, ghost zones included (strides from chemora_grid_layout); a state
 *    of nvars variables is nvars such arrays back to back.  The grid is
 *    periodic: point i sits at x = i*dx, i = 0..n-1.
 *  - `stream` is a cudaStream_t; NULL is the legacy default stream.  Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - Every call returns a status (CHEMORA_OK or a negative code).  Errors
 *    never abort the process and never trap the GPU; chemora_last_error()
 *    returns a message for the calling thread.
 *  - Not thread-safe per handle: one handle is used by one host thread at a
 *    time.
 */
#ifndef CHEMORA_H
#define CHEMORA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  CHEMORA_OK = 0,
  CHEMORA_EINVAL = -1,      /* bad argument (size, pointer, kind, mode) */
  CHEMORA_ENOMEM = -2,      /* device or host allocation failed */
  CHEMORA_ECUDA = -3,       /* a CUDA runtime call or launch failed */
  CHEMORA_ETIMEOUT = -4,    /* a bounded device-side wait gave up */
  CHEMORA_ENONFINITE = -5,  /* NaN/Inf detected where checked */
  CHEMORA_EUNSUPPORTED = -6 /* valid request this build does not serve */
};

enum {
  CHEMORA_WAVE = 1,      /* u_t = rho, rho_t = Lap u (2 vars, ghosts >= 2) */
  CHEMORA_WAVE_VARC = 2, /* u_t = rho, rho_t = s Lap u + grad s . grad u,
                            s = c^2 (2 vars + coefficient, ghosts >= 2) */
  CHEMORA_BSSN = 3,      /* BSSN phi-form, 24 vars, ghosts >= 3 */
  CHEMORA_WAVE1 = 4      /* first-order form of Eq. 1: u_t = rho,
                            rho_t = sum_i D_i v_i, (v_i)_t = D_i rho
                            (5 vars u, rho, v_x, v_y, v_z; ghosts >= order/2) */
};

/* BSSN variable order: 0 phi; 1-6 gt_ij (xx,xy,xz,yy,yz,zz); 7 K;
 * 8-13 At_ij (same order); 14-16 Xt^i; 17 alpha; 18-20 beta^i; 21-23 B^i. */

typedef struct {
  double eps_diss; /* Kreiss-Oliger strength (BSSN), default 0.1 */
  double eta;      /* Gamma-driver damping (BSSN), default 2 */
  int slicing;     /* 0: 1+log, 1: harmonic, 2: frozen lapse */
  int shift;       /* 0: Gamma-driver, 1: frozen shift and B */
  int fd_order;    /* finite-difference order: 0 = 4; CHEMORA_WAVE and
                      CHEMORA_WAVE1 accept 2, 4, 6, 8 (Sec. 3.2.2, operators
                      of arbitrary order; ghosts >= order/2), the other
                      systems 4 only */
} chemora_params;

typedef struct chemora_grid chemora_grid;
typedef struct chemora_system chemora_system;
typedef struct chemora_batch chemora_batch;
typedef struct chemora_amr chemora_amr;

/* Uniform grid of nx*ny*nz interior points, nghost ghost layers on each face,
 * spacing dx, for states of nvars grid functions (Sec. 2: the driver's grid
 * with ghost zones).  Errors: EINVAL if a size is < 1, nghost < 1, nvars < 1,
 * dx <= 0, the state exceeds 2^40 doubles, or out is NULL. */
int chemora_grid_create(int nx, int ny, int nz, int nvars, int nghost, double dx,
                        chemora_grid** out);

/* Strides in doubles: sy between y-neighbours, sz between z-neighbours, svar
 * between variables (x stride is 1); any output pointer may be NULL. */
int chemora_grid_layout(const chemora_grid* grid, int64_t* sy, int64_t* sz, int64_t* svar);

/* A PDE system on a grid (Sec. 3.2.1: the physics description).  kind is
 * CHEMORA_WAVE, CHEMORA_WAVE_VARC, CHEMORA_BSSN or CHEMORA_WAVE1; params may
 * be NULL for the defaults (eps 0.1, eta 2, 1+log, Gamma-driver, order 4);
 * the wave systems read only fd_order.  The grid must outlive the system.  Scratch for RK4 (three states)
 * is allocated on first use.  Errors: EINVAL for a wrong nvars/nghost for the
 * kind or bad params, ENOMEM. */
int chemora_system_create(chemora_grid* grid, int kind, const chemora_params* params,
                          chemora_system** out);

/* Set the coefficient s = c^2 of CHEMORA_WAVE_VARC from the wave speed c (one
 * grid function, interior read, ghosts ignored): the library keeps its own
 * copy with periodic ghosts, and its 4th-order centred derivatives D_d s,
 * taken once here because the speed does not change in time (the right-hand
 * side s Lap u + sum_d D_d s D_d u reads them at the point).  Synchronous
 * with respect to `stream`.
 * Errors: EINVAL for another kind or NULL c. */
int chemora_system_set_speed(chemora_system* sys, const double* c, void* stream);

/* Periodic ghost zones of all variables of `state`, in place (Sec. 2, ghost
 * zones; the periodic image of the interior). */
int chemora_fill_ghosts(chemora_system* sys, double* state, void* stream);

/* Periodic ghost zones along the axes in the bit mask `axes` (1 x, 2 y,
 * 4 z) only: a ghost point takes the value of the point with its
 * coordinates wrapped along those axes; layers outside the interior along
 * the other axes are left as they are (for a domain split along z, exchange
 * the z halos first, then fill x and y).  axes = 7 equals
 * chemora_fill_ghosts. */
int chemora_fill_ghosts_axes(chemora_system* sys, double* state, int axes, void* stream);

/* rhs <- RHS(state) on the interior (Sec. 3.2: the "RHS" calculation).  The
 * ghosts of state must be valid; the ghosts of rhs are left untouched.
 * state and rhs must not overlap. */
int chemora_rhs(chemora_system* sys, const double* state, double* rhs, void* stream);

/* nsteps classic RK4 steps of size dt, in place (Sec. 2, time integrator).
 * Fills ghosts itself before every stage and on return.  Each stage is one
 * fused kernel (stencils + RHS + Runge-Kutta update).  For nsteps >= 2 one
 * step is captured in a CUDA graph (cached per state pointer, dt and launch
 * shape) and replayed; plain launches are used while profiling is enabled
 * or when the caller's stream is itself being captured.  Errors: EINVAL for
 * nsteps < 0 or a non-finite dt. */
int chemora_rk4_step(chemora_system* sys, double* state, double dt, int nsteps, void* stream);

/* One fused stage kernel (stencils + RHS + Runge-Kutta update), the
 * building block of chemora_rk4_step for drivers that own their ghost
 * zones (e.g. a domain split across GPUs).  With k = RHS(src) on the interior:
 *   mode 0: dst = k
 *   mode 1: acc = k;        dst = yn + c2 k
 *   mode 2, 3: acc += 2 k;  dst = yn + c2 k
 *   mode 4: dst = yn + c1 (acc + k)
 * so one classic RK4 step is modes 1-4 with (c2 = dt/2, dt/2, dt; c1 =
 * dt/6), each preceded by filling the ghosts of its src.  The ghosts of src
 * must be valid; src must not overlap dst, acc or yn's written interior. */
int chemora_stage(chemora_system* sys, int mode, const double* src, const double* yn, double* acc,
                  double* dst, double c1, double c2, void* stream);

/* chemora_rk4_step for a state in HOST memory (pinned memory recommended):
 * the state is copied to a library-owned device buffer, advanced nsteps RK4
 * steps, and copied back.  Synchronous with respect to `stream`.  This is the
 * end-to-end call for callers that keep their data on the host. */
int chemora_rk4_step_host(chemora_system* sys, double* host_state, double dt, int nsteps,
                          void* stream);

/* chemora_rk4_step without any device allocation, for callers that cannot
 * call cudaMalloc (allocator hooks and host callbacks, frameworks that must
 * account for every device allocation, real-time loops that may not risk an
 * allocation failing or synchronising mid-run).  The paper has no
 * counterpart; it is a deployment variant of chemora_rk4_step with the same
 * arguments.  It always launches the ahead-of-time default stage kernel, so
 * its results agree with chemora_rk4_step's to rounding (chemora_rk4_step may
 * run an autotuned or run-time specialised kernel).
 * Scratch: a fixed 32 MiB array (4,194,304 doubles) compiled into the
 * library; it fits states with nvars*(nx+2g)*(ny+2g)*(nz+2g) <= 1,398,101
 * doubles (e.g. the wave equation on 84^3 padded points, BSSN on 38^3),
 * larger ones return CHEMORA_EINVAL.  The first call on a device looks up the
 * array's device address, which makes the CUDA driver load the array's
 * module and reserve its 32 MiB on that device (held until the process
 * exits); if the device has no room that first call returns CHEMORA_ENOMEM.
 * Make the first call before any stream capture.  All calls share the array:
 * calls that overlap on the GPU race and must be serialised by the caller. */
int chemora_rk4_step_noalloc(chemora_system* sys, double* state, double dt, int nsteps,
                             void* stream);

/* BSSN constraints on the interior (analysis; the oracle's convergence
 * measures): out holds 7 grid functions laid out like the state --
 * 0: Hamiltonian H = R + 2/3 K^2 - At_ij At^ij;
 * 1-3: momentum M^i = d_j At^ij + Gamma~^i_jk At^jk + 6 At^ij d_j phi
 *      - 2/3 gt^ij d_j K; 4-6: Gamma constraint G^i = Xt^i - gt^jk Gamma~^i_jk.
 * The ghosts of state must be valid; ghosts of out are untouched.
 * Errors: EINVAL for a non-BSSN system. */
int chemora_constraints(chemora_system* sys, const double* state, double* out, void* stream);

/* Discrete energy of the scalar wave equation, E = 1/2 sum (rho^2 - u Lap_h u)
 * h^3 over the interior (the "Energy" calculation of Fig. 2, in the
 * two-variable form; conserved by the semi-discrete system, non-increasing
 * under RK4).  The ghosts of state must be valid.  *energy is a HOST double;
 * the reduction order is fixed, so the result is deterministic.
 * Synchronous.  Errors: EINVAL for another kind. */
int chemora_energy(chemora_system* sys, const double* state, double* energy, void* stream);

/* NaN/Inf sentinel: counts the non-finite interior values of `state` into
 * *nonfinite (HOST, may be NULL) and returns CHEMORA_ENONFINITE if there are
 * any.  Synchronous.  (Failure detection; no counterpart in the paper.) */
int chemora_check_finite(chemora_system* sys, const double* state, int64_t* nonfinite, void* stream);

/* Batched patches (Sec. 4: AMR / multi-block drivers advance many patches):
 * npatch independent periodic grids, patch p of dims[3p..3p+2] = (nx,ny,nz)
 * interior points, one spacing dx, nghost ghosts, all of `kind` (CHEMORA_BSSN
 * or CHEMORA_WAVE).  Storage for every patch's state is library-owned and
 * contiguous.  Errors: EINVAL for npatch < 1, a size < 1 or an unsupported
 * kind; ENOMEM. */
int chemora_patches_create(int npatch, const int* dims, int nghost, double dx, int kind,
                           const chemora_params* params, chemora_batch** out);

/* Device pointer to patch p's state inside the batch storage (layout as for
 * a grid of that patch's dims); valid until the batch is destroyed. */
int chemora_patches_state(chemora_batch* batch, int p, double** dev_ptr);

/* nsteps RK4 steps of every patch.  mode 0: per stage one batched ghost-fill
 * launch and one persistent launch that pulls (patch, tile) work items from a
 * work-list, the whole step captured once in a CUDA graph and replayed;
 * mode 1: per patch and stage separate launches (the reference schedule).
 * Errors: EINVAL for a bad mode or a corrupted work-list, ETIMEOUT if a
 * persistent stage launch passed the time limit set with
 * chemora_patches_set_time_limit (the batch state is then undefined). */
int chemora_patches_step(chemora_batch* batch, double dt, int nsteps, int mode, void* stream);

/* Time limit of each persistent stage launch of chemora_patches_step mode 0
 * (failure detection; no counterpart in the paper).  A block of the
 * persistent kernel takes no further work item once `seconds` of SM clock
 * cycles, counted at the device's peak clock, have passed since it started;
 * the step then returns CHEMORA_ETIMEOUT and the context stays usable.
 * seconds <= 0 removes the limit (the default).  A change takes effect at
 * the next step (the step graph is captured again).  Errors: EINVAL for a
 * bad handle or a non-finite value. */
int chemora_patches_set_time_limit(chemora_batch* batch, double seconds);

/* Failure injection for tests (no counterpart in the paper): overwrite work
 * item `item` of the batch's device work-list with an entry naming a patch
 * outside the patch table.  The persistent kernel checks every item before
 * touching memory, skips such an item and sets a device error word, so the
 * next chemora_patches_step(mode 0) returns CHEMORA_EINVAL instead of
 * faulting.  The batch stays corrupted; destroy it afterwards. */
int chemora_patches_inject_fault(chemora_batch* batch, int item);

/* Two-level mesh refinement with Berger-Oliger subcycling (Sec. 4: the AMR
 * driver refines patches and subcycles them in time) for the scalar wave
 * (CHEMORA_WAVE) or the BSSN system (CHEMORA_BSSN, with `params`, NULL for
 * the defaults), 4th order.  Level 0: periodic grid of nc[0] x nc[1] x nc[2]
 * points (x, y, z), spacing dx, r ghost layers (r = 2 for the wave, 3 for
 * BSSN: the stencil radius).  Level 1: nbox disjoint boxes; box b refines the
 * coarse points [lo[3b+d], hi[3b+d]) along axis d by 2 (2 (hi - lo) fine
 * points, spacing dx/2) and carries a buffer zone of B = 4 r points around
 * its interior (8 for the wave, 12 for BSSN).  The prolongation of a buffer
 * reads M = B/2 + 2 coarse points beyond the box, so each box must satisfy
 * M - r <= lo < hi <= nc + r - 1 - M per axis (wave: 4 <= lo, hi <= nc - 5;
 * BSSN: 5 <= lo, hi <= nc - 6).  Storage is library-owned; all boxes are
 * advanced together by one batched stage launch per fine RK stage.
 * Errors: EINVAL (kind, extents, boxes out of range or overlapping, params,
 * fd order other than 4), ENOMEM. */
int chemora_amr_create_boxes(int kind, const int* nc, int nbox, const int* lo, const int* hi, double dx,
                             const chemora_params* params, chemora_amr** out);

/* The single-box scalar-wave case of chemora_amr_create_boxes: an nc^3
 * coarse grid and the box [lo[d], hi[d]), 4 <= lo[d] < hi[d] <= nc - 5. */
int chemora_amr_create(int nc, const int* lo, const int* hi, double dx, chemora_amr** out);

/* Device pointer and strides (doubles) of level 0 (the coarse grid, r
 * ghosts) or 1 + b (box b, padded by its buffer B) of the state.  Fine index
 * B + f along axis d of box b is the fine point of global fine index
 * 2 lo[3b+d] + f (f = 0 .. 2 (hi - lo) - 1); the buffer layers hold the last
 * prolongation after a step.  Any output may be NULL.  Errors: EINVAL. */
int chemora_amr_state(chemora_amr* amr, int level, double** dev_ptr, int64_t* sy, int64_t* sz,
                      int64_t* svar);

/* nsteps coarse steps of size dt.  Per step: the coarse level takes one RK4
 * step (periodic ghosts); every box takes two RK4 steps of dt/2, its buffer
 * filled at the start of each by quintic Lagrange prolongation of coarse
 * data interpolated in time with cubic Hermite through the coarse state and
 * right-hand side at t_n and t_{n+1}, its RK stages evaluated on the
 * interior extended into the buffer (stage s on the interior extended by
 * B - r s: the valid region shrinks by the stencil radius per stage); then
 * the fine values are injected into the coincident coarse points and the
 * coarse ghosts refilled.  mode 0: each fine RK stage of all boxes is one
 * persistent launch over a work-list of every box; mode 1: the single-grid
 * stage kernel box by box (same results to rounding; for comparison).  The
 * caller sets the coarse interior and the box interiors before the first
 * step.  Mode 0 synchronises `stream` at the end (it reads the batched
 * kernel's error word).  Errors: EINVAL, ECUDA. */
int chemora_amr_step_mode(chemora_amr* amr, double dt, int nsteps, int mode, void* stream);

/* Pick the launch shape of the coarse level's stage kernel by timing the
 * plausible ones on the coarse state (as chemora_autotune does for a
 * system); the fine boxes always run the batched work-list kernel.  Fills
 * the coarse ghosts; the coarse RK scratch is overwritten.  *variant may be
 * NULL.  Synchronous.  Errors: EINVAL, ECUDA. */
int chemora_amr_autotune(chemora_amr* amr, int* variant, void* stream);

/* chemora_amr_step_mode with mode 0. */
int chemora_amr_step(chemora_amr* amr, double dt, int nsteps, void* stream);

/* Discrete adjoint of the variable-speed wave equation under RK4 (the exact
 * transpose of the fully discrete map; the paper's Kranc mentions generated
 * Jacobians in Sec. 3.2.1 -- this is the reverse-mode counterpart).
 *   forward:  state0 (2 vars) advanced nsteps RK4 steps of size dt with
 *             s = c^2 (c: one grid function, interior read);
 *   loss:     J = 1/2 sum_r (u_N[recv_idx[r]] - data[r])^2, recv_idx padded
 *             linear indices into one grid function (interior points),
 *             HOST arrays, nrecv >= 1; *loss is written on the host;
 *   gradient: grad_state0 (2 vars) = dJ/dstate0, grad_c = dJ/dc = 2 c sbar,
 *             interior written, ghosts zero.
 * Checkpoints of the state are kept every ckpt_every steps (device memory
 * owned by the library) and each segment is recomputed in reverse order.
 * Synchronous with respect to `stream` (the loss is returned).  Errors: EINVAL
 * for another kind, nsteps < 1, ckpt_every < 1, a receiver outside the
 * interior. */
int chemora_adjoint_rk4(chemora_system* sys, const double* state0, const double* c, double dt,
                        int nsteps, int ckpt_every, const int64_t* recv_idx, int nrecv,
                        const double* data, double* loss, double* grad_state0, double* grad_c,
                        void* stream);

/* Autotuner (the paper's run-time library auto-tunes the thread assignment,
 * Sec. 3.2.3): ranks the compiled launch shapes of the system's stage kernel
 * with a model of idle edge threads and wave quantisation, times the
 * plausible ones on `state` (its ghosts are filled first) and keeps the
 * fastest for this system.  Shapes of the same body perform the same
 * per-point arithmetic; the lane-, shared-memory- and z-queue-sharing bodies
 * form the stencils' differences in another order, so results of different
 * bodies agree to rounding (each within the parity tolerances of the
 * oracle).  *variant and *best_ms (time of a middle RK stage of the winner)
 * may be NULL.  For the order-4 scalar wave it also times whole RK4 steps
 * (on a copy of `state`) with the per-stage kernels and with the
 * launch-chained path of chemora_system_set_chain, and keeps the faster.
 * Synchronous. */
int chemora_autotune(chemora_system* sys, double* state, int* variant, double* best_ms, void* stream);

/* Launch-chained RK4 steps for the order-4 scalar wave (CHEMORA_WAVE, Sec. 3
 * Eq. 1; a runtime choice of this library, no counterpart in the paper):
 * with mode 1, chemora_rk4_step runs each stage as a kernel that reads the
 * neighbours at their periodic images (no ghost fill between stages) and is
 * chained to the previous stage by a programmatic dependent launch, 8 steps
 * per captured CUDA graph, and fills the ghosts once at the end; results are
 * bit-equal to the per-stage kernels.  It pays off on small grids, where the
 * per-stage launches and ghost fills are latency-bound (chemora_autotune
 * picks it by timing).  Not used while the stream is being captured or
 * profiling is on.  mode: 0 per-stage kernels, 1 launch-chained, -1 query
 * only; *active (may be NULL) receives the mode in force.  Errors: EINVAL,
 * EUNSUPPORTED (another kind or order). */
int chemora_system_set_chain(chemora_system* sys, int mode, int* active);

/* Number of compiled launch shapes of the stage kernel of `kind`. */
int chemora_variant_count(int kind);

/* Launch shape `variant` of the stage kernel of `kind`: block tx x ty
 * threads, min_blocks resident blocks per SM asked of the compiler (the
 * register cap), and sharing: 0 the direct body (neighbours through the
 * read-only cache), 1 x-direction work shared across warp lanes (needs
 * nx % tx == 0 and 3 ghost layers), 2 in addition y-direction differences
 * and z-derivative rows shared through shared memory (any ny), 4 (scalar
 * wave, order 4) x-direction work shared across warp lanes and each thread
 * marching along z with a register queue of z first differences (needs
 * nx % tx == 0).  A shape whose condition fails on a grid runs as shape 0.  Outputs may be NULL;
 * CHEMORA_EINVAL for an unknown kind or index. */
int chemora_variant_info(int kind, int variant, int* tx, int* ty, int* min_blocks, int* sharing);

/* Query (set < 0) or set (set = index) the launch shape of a system; tx, ty
 * receive the block shape.  Any output may be NULL. */
int chemora_system_variant(chemora_system* sys, int set, int* variant, int* tx, int* ty);

/* Run-time specialisation of the stage kernel (Sec. 3.2.3: the run-time
 * library compiles loop kernels once parameter values are known, to cut code
 * and register overhead).  With enable = 1 the library writes a CUDA source
 * that instantiates the body of the system's current launch shape with the
 * grid extents, ghost width and strides as literals, the scalars 1/(12h),
 * 1/(12h^2), 1/(144h^2), the dissipation scale and the gauge parameters as
 * compile-time constants (exact hexadecimal literals: same arithmetic as the
 * ahead-of-time kernel) and one kernel per Runge-Kutta stage mode; compiles
 * it with NVRTC (loaded with dlopen; libnvrtc.so.13) for the device's
 * architecture; loads the cubins; and from then on chemora_rhs,
 * chemora_stage and chemora_rk4_step launch these kernels.  The
 * specialisation belongs to the launch shape it was built for: after
 * chemora_system_variant or chemora_autotune selects another shape the
 * ahead-of-time kernels run until chemora_system_specialize is called
 * again.  enable = 0 returns to the ahead-of-time kernels (the compiled
 * kernels are kept for a later enable = 1).
 *
 * cache_dir: directory for compiled cubins, created if missing, keyed by a
 * hash of the kernel source, the device headers it includes, the options
 * and the NVRTC version; NULL means $CHEMORA_JIT_CACHE,
 * else $HOME/.cache/chemora_jit; "" disables the disk cache.  A cache that
 * cannot be written is skipped silently.  *compile_seconds (may be NULL)
 * receives the wall time of the compilation, 0 when every cubin came from
 * the cache or nothing had to be built.  Synchronous; drops the system's
 * captured RK4 step graph.  Errors: CHEMORA_EUNSUPPORTED when NVRTC cannot
 * be loaded or the system is not BSSN (only BSSN is specialised);
 * CHEMORA_ECUDA when compilation or loading fails (the compiler log heads
 * chemora_last_error) -- the system then keeps its ahead-of-time kernels.
 * No device memory is allocated beyond the loaded code. */
int chemora_system_specialize(chemora_system* sys, int enable, const char* cache_dir,
                              double* compile_seconds);

/* Per-system kernel timing: when enabled, every RHS/RK-stage launch of the
 * system is bracketed by CUDA events on its stream.  chemora_profile_read
 * synchronises those events and returns the summed device time (ms) and the
 * number of timed launches since the last reset. */
int chemora_profile_enable(chemora_system* sys, int on);
int chemora_profile_read(chemora_system* sys, double* total_ms, int64_t* launches, int reset);

/* Number of kernels this library has launched in this process so far. */
int64_t chemora_launch_count(void);

/* Operation counts of one RHS evaluation per interior point for `kind`, as
 * counted by the kernel generator on the expression DAG it emitted: fp64
 * instructions (add/sub/mul/fma each 1) and algorithmic flops (fma 2,
 * add/sub/mul/exp/reciprocal 1). */
int chemora_opcount(int kind, int64_t* fp64_instructions, int64_t* flops);

/* Operation counts per interior point of one RHS evaluation by the body the
 * system currently launches (the autotuned launch shape may use a body that
 * shares x-direction work across warp lanes, y differences through shared
 * memory, or z differences through a register queue; the counts then
 * include, per point, that sharing's own work).  Counts as
 * chemora_opcount. */
int chemora_system_opcount(chemora_system* sys, int64_t* fp64_instructions, int64_t* flops);

/* Measure the device's FP64 fused-multiply-add throughput (flop/s, fma = 2)
 * with a short kernel of independent FMA chains on every SM (measurement
 * support for the roofline; no counterpart in the paper).  Synchronous. */
int chemora_fp64_peak(double* flops_per_s, void* stream);

/* Message for the last error on the calling thread ("" if none). */
const char* chemora_last_error(void);

/* Release a grid, system, batch or refinement handle (NULL is ignored).  A
 * grid must be released after the systems that use it. */
void chemora_destroy(void* handle);

#ifdef __cplusplus
}
#endif

#endif /* CHEMORA_H */
