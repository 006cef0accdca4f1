/*
 * microsim_gb.h -- C ABI of the GB300 grand-potential phase-field step library.
 *
 * The library advances the multi-phase, multi-component grand-potential model
 * of the MICROSIM paper (arXiv 2404.01035, Sec. 2.1 "Grand-potential
 * formulation", Sec. 3 "Thermodynamic coupling") by explicit finite-difference
 * time steps on a 2-D or 3-D grid.  One step computes, per cell:
 *   - the anisotropic gradient-energy divergence div(da/dgrad phi_a) and the
 *     centre term da/dphi_a (Eqs. Eqn_a, aniso_eqn, four-fold a_c),
 *   - the obstacle or well potential derivative (Eqs. Obstacle, Well),
 *   - the driving force dpsi/dphi_a = sum_b psi^b dh_b/dphi_a (Eq. hphi) with
 *     parabolic free energies (Eqs. free_energy_density, Coeff_B, Coeff_C),
 *   - the phi update of Eq. (phi_eqn) with the Lagrange multiplier realised
 *     as the Euclidean projection onto the simplex (obstacle) or onto the
 *     sum-one hyperplane (well),
 *   - the chemical-potential update of Eq. (Mu_explicit_temperature) with
 *     mobility M = sum_a h_a D^a chi^a and a frozen, pulled temperature field.
 * Every step runs in hand-written sm_103a CUDA kernels; there is no CPU path.
 *
 * Conventions
 *   - Field arrays exchanged with the caller are dense, row-major
 *     [field][z][y][x] (x fastest), nz = 1 for 2-D grids, in the context's
 *     dtype (float for MS_F32, double for MS_F64).  phi holds N fields,
 *     mu holds K-1 fields (K = number of components).
 *   - Phase N-1 is the liquid, the reference phase of the parabolic free
 *     energies (B^l = C^l = 0).
 *   - Every call returns ms_status; no exception crosses the ABI.  The text of
 *     the last error of a context is returned by ms_last_error(ctx); errors
 *     raised before a context exists are returned by ms_last_error(NULL)
 *     (thread-local).
 *   - Device-side faults (non-finite values, barrier timeouts) are recorded in a
 *     sticky device status word that ms_sync / ms_diag / ms_grad read.
 *   - All work is enqueued on the stream given at creation; calls return once
 *     the work is enqueued unless stated otherwise.
 *   - Buffers handed in are only read during the call (copied); the library
 *     owns its device state and releases it in ms_destroy.
 */
#ifndef MICROSIM_GB_H
#define MICROSIM_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms_ctx ms_ctx;
typedef struct ms_batch ms_batch;

typedef enum {
  MS_OK = 0,
  MS_ERR_ARG = 1,          /* invalid argument or unsupported combination */
  MS_ERR_CUDA = 2,         /* a CUDA runtime/driver call failed */
  MS_ERR_OOM = 3,          /* device allocation failed */
  MS_ERR_DT_UNSTABLE = 4,  /* dt above the explicit stability bound */
  MS_ERR_NONFINITE = 5,    /* NaN/Inf found in the state (sticky) */
  MS_ERR_TIMEOUT = 6,      /* a bounded device wait gave up (sticky) */
  MS_ERR_BOUNDS = 7,       /* size beyond a fixed library limit */
  MS_ERR_STATE = 8,        /* call not valid in the context's current state */
  MS_ERR_UNSUPPORTED = 9   /* (dim, phases, components, dtype) not compiled in */
} ms_status;

typedef enum { MS_F32 = 0, MS_F64 = 1 } ms_dtype;

/* Boundary codes of the paper's BOUNDARY key (Sec. "Input files"):
 * 1 = Neumann (no-flux, mirror ghost cell), 3 = periodic. */
enum { MS_BC_NOFLUX = 1, MS_BC_PERIODIC = 3 };
/* Library code (not a paper code) for the z faces of a 3-D sub-domain whose
 * ghost planes are filled by ms_halo_exchange / ms_halo_mirror (slab
 * decomposition of one domain into several contexts). */
enum { MS_BC_HALO = 16 };

/* Function_W: 1 = multi-obstacle (Eq. Obstacle), 2 = multi-well (Eq. Well). */
enum { MS_POT_OBSTACLE = 1, MS_POT_WELL = 2 };

/* Grid: DIMENSION, MESH_X/Y/Z, DELTA_X and BOUNDARY per axis. */
typedef struct {
  int dim;          /* 2 or 3 */
  int nx, ny, nz;   /* cells per axis; nz is ignored (taken as 1) for dim = 2 */
  double dx;        /* cell size (DELTA_X = DELTA_Y = DELTA_Z) */
  int bc[3];        /* MS_BC_* for the x, y, z axes (both faces of an axis) */
  int z_origin;     /* lab index of this grid's first cell along the last axis
                       (z in 3-D, y in 2-D): the first plane of a slab of a
                       larger domain, or the frame offset after ms_shift (0
                       otherwise); the temperature field and the phi-noise
                       counter use lab indices */
} ms_grid;

/* Model inputs, named after the paper's infile keys.  All pointers are host
 * arrays of doubles read during the call.  N = phases, M = K-1 solutes. */
typedef struct {
  ms_dtype dtype;          /* arithmetic type of the state and the step */
  int potential;           /* MS_POT_OBSTACLE or MS_POT_WELL (Function_W) */
  double eps;              /* epsilon: interface-width parameter */
  double tau;              /* tau: relaxation constant; phase mobility is 1/tau */
  double dt;               /* DELTA_t */
  const double* gamma;     /* [N][N] GAMMA, symmetric */
  const double* delta;     /* [N][N] dab, anisotropy strength; 0 = isotropic pair */
  const double* rot;       /* [N][N][3][3] Rotation_matrix per pair; NULL = identity.
                              2-D grids use the upper-left 2x2 block. */
  const double* gamma3;    /* [N][N][N] Gamma_abc, symmetric; NULL = none */
  const double* D;         /* [N][M][M] DIFFUSIVITY matrices */
  const double* A;         /* [N][M][M] parabolic coefficients A_ij, i <= j used */
  const double* ceq;       /* [N][M] equilibrium compositions at T_ref (ceq) */
  const double* slopes;    /* [N][M] d c_eq / dT (slopes) */
  const double* f0;        /* [N] constant added to f^a (isothermal drive); NULL = 0 */
  double T_ref;            /* temperature at which ceq is given */
  double T0, G, z0, V;     /* Tempgrady: T(s,t) = T0 + G (s - z0 - V t), s the
                              cell-centre coordinate along the last axis */
  double t0;               /* physical time of the initial state */
  double noise_amp;        /* Noise_phasefield / Amp_Noise_Phase: every step adds
                              dt * noise_amp * xi to the phi rate of each phase a
                              with 0 < phi_a < 1 at the cell, before the
                              projection; xi uniform in [-1/2, 1/2) from the
                              SplitMix64 finaliser (Steele, Lea, Flood 2014)
                              applied to noise_seed, the step index and the lab
                              cell index x + nx (y + ny z) times N plus a.  0 =
                              off.  Not available with ms_grad or ms_batch_*. */
  unsigned long long noise_seed;
  int anti_trapping;       /* 1 = anti-trapping current j_at (Sec. 2.1, Eq. jatr;
                              obstacle or well form by `potential`) inside the
                              divergence of the mu update, for the liquid =
                              phase N-1; each step then runs a second kernel
                              that corrects mu with phi^{n+1} of the
                              neighbours.  0 = off.  Not available with
                              ms_grad, ms_batch_* or MS_BC_HALO faces. */
  int grain_growth;        /* GRAINGROWTH = 1 (Sec. 4 "Grain-growth"): the phi
                              equation without the chemical term dpsi/dphi, mu
                              held (copied unchanged every step); the fields
                              keep their layout (N grains, M >= 1 mu fields that
                              stay constant).  Not available with
                              anti_trapping, ms_grad or ms_batch_*. */
  const double* elastic_C; /* Elasticity (Sec. 2 "Elasticity implementation",
                              homogeneous stiffness): 6 x 6 Voigt stiffness,
                              order xx yy zz yz xz xy, engineering shear; NULL =
                              off.  Before every step the periodic equilibrium
                              strain of the eigenstrain sum_a eps*^a h_a(phi) is
                              solved by FFT (cuFFT, opened at run time; zero
                              mean strain), and -sigma : eps*^b joins each
                              phase potential.  2-D grids use plane strain.
                              Needs periodic boundaries and N in {2, 3, 8}; not
                              available with grain_growth, ms_grad, ms_batch_*
                              or MS_BC_HALO faces. */
  const double* eigenstrain; /* [N][3][3] eigenstrain of each phase (symmetric
                              tensor components), read with elastic_C. */
} ms_params;

/* Optional device allocator (e.g. a framework's caching allocator).  NULL in
 * ms_create means cudaMalloc / cudaFree.  alloc returns NULL on failure. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*release)(void* ptr, void* user);
  void* user;
} ms_allocator;

/* Create a context: validates the inputs, derives the per-phase parabolic
 * coefficients B^a(T), C^a(T), chi^a = (Hessian of f^a)^-1 (Eqs. Coeff_B,
 * Coeff_C; the off-diagonal sum of Coeff_B taken with the sign its own equal-mu
 * condition gives), checks dt against the explicit stability bound (FP64,
 * MS_ERR_DT_UNSTABLE when above it), allocates the ping-pong device state and
 * enqueues nothing.  stream is a cudaStream_t (NULL = legacy default stream).
 * n_phases in [2, 8], n_components in [2, 4].  Returns MS_ERR_UNSUPPORTED when
 * the (dim, N, K, dtype) step kernel is not compiled into the library. */
ms_status ms_create(const ms_grid* grid, int n_phases, int n_components,
                    const ms_params* params, void* stream, const ms_allocator* alloc,
                    ms_ctx** out);

/* The checks of ms_create without a device: the inputs, the derived
 * coefficients and the compiled (dim, N, K, dtype) kernels, with the same
 * status codes.  *dt_bound (may be NULL) receives the explicit stability
 * bound on dt, (dx^2 / 2 dim) min(tau / (gamma_max (1 + 15 delta_max)),
 * 1 / max_a ||chi^a^-1 D^a chi^a||_inf), whenever the checks before it pass,
 * also when dt exceeds it (MS_ERR_DT_UNSTABLE).  Allocates nothing and
 * touches no GPU. */
ms_status ms_check_params(const ms_grid* grid, int n_phases, int n_components,
                          const ms_params* params, double* dt_bound);

/* Release all device and host resources (synchronises the stream first). */
void ms_destroy(ms_ctx* ctx);

/* Text of the last error on ctx (or of the calling thread when ctx is NULL). */
const char* ms_last_error(const ms_ctx* ctx);

/* Replace the model parameters (dt, eps, tau, delta, D, ...); grid, N, K and
 * dtype must be unchanged.  Turning on the anti-trapping current or
 * elasticity allocates their buffers (and FFT plans) here; if that fails the
 * call returns the error and the context keeps the parameters it had.  While
 * adjoint checkpoints are recording, phi noise, the anti-trapping current,
 * grain growth and elasticity cannot be turned on (MS_ERR_UNSUPPORTED), and
 * a successful update drops the snapshots recorded so far: the recording
 * restarts at the current step, so that ms_grad never mixes two parameter
 * sets. */
ms_status ms_update_params(ms_ctx* ctx, const ms_params* params);

/* Copy the state in.  phi: N fields, mu: K-1 fields, dense [f][z][y][x] in
 * the context dtype; on_device = 1 if the pointers are device pointers, 0 for
 * host memory (pinned or pageable).  Resets the step counter to 0 and the time
 * to params->t0, and clears recorded adjoint checkpoints. */
ms_status ms_set_fields(ms_ctx* ctx, const void* phi, const void* mu, int on_device);

/* Copy the current state out (same layout as ms_set_fields); synchronous. */
ms_status ms_get_fields(ms_ctx* ctx, void* phi, void* mu, int on_device);

/* Borrowed device views of the current state: *phi_dev / *mu_dev point at
 * cell (0,0,0) of field 0; element (f,z,y,x) is at
 * base + f*strides[0] + z*strides[1] + y*strides[2] + x*strides[3] (elements).
 * Valid until the next ms_step / ms_set_fields / ms_destroy. */
ms_status ms_fields(ms_ctx* ctx, void** phi_dev, void** mu_dev, int64_t strides[4]);

/* Enqueue n explicit steps (each a single fused kernel launch) and, every
 * diag_every steps (ms_set_diag_every), the FP64 diagnostics kernel. */
ms_status ms_step(ms_ctx* ctx, int64_t n);

/* Run FP64 diagnostics of the current state and wait for them:
 * out[0..K-2]   sum over cells of c_i = sum_a h_a c^a_i(mu, T)  (solute mass)
 * out[K-1]      max |sum_a phi_a - 1|
 * out[K]        min phi,   out[K+1] max phi
 * out[K+2]      number of non-finite values in the state
 * out[K+3]      max over cells of the explicit mu-diffusion number
 *               dt * sum_faces max_i sum_j |(chi^-1 M_f)_ij| / dx^2
 *               (the forward-Euler diffusion update is stable when <= 1)
 * out[K+4]      step count,  out[K+5] physical time
 * Also returns MS_ERR_NONFINITE when non-finite values are present. */
ms_status ms_diag(ms_ctx* ctx, double* out);
#define MS_DIAG_LEN(K) ((K) + 6)

/* Run the diagnostics every k steps inside ms_step (0 = never, default). */
ms_status ms_set_diag_every(ms_ctx* ctx, int64_t k);

/* Wait for the stream; returns the sticky device status (MS_OK,
 * MS_ERR_NONFINITE or MS_ERR_TIMEOUT). */
ms_status ms_sync(ms_ctx* ctx);

/* Failure-path self-test (the paper has no counterpart; a library service
 * for callers that want to see the timeout path work).  Enqueues one small
 * kernel whose single thread waits, through the same bounded mbarrier wait
 * the step kernels use, on a barrier that nothing completes, with a limit of
 * limit_ns nanoseconds of %globaltimer (1e3 <= limit_ns <= 1e9); the wait
 * gives up, records the timeout in the context's sticky status word and the
 * kernel returns (no copy is in flight).  ms_sync / ms_diag then return
 * MS_ERR_TIMEOUT for the rest of the context's life; the CUDA context stays
 * usable for other ms contexts.  The step kernels' own waits keep their
 * fixed one-second limit.  MS_ERR_ARG for a limit outside the range. */
ms_status ms_selftest_timeout(ms_ctx* ctx, int64_t limit_ns);

/* FP32 arithmetic peak of the current device in TFLOP/s, measured (the paper
 * has no counterpart; a measurement service for the ALU roof of the step's
 * roofline): a grid of 64 warps per SM, each thread 8 independent chains of
 * fused multiply-adds, scalar (paired = 0) or two-lane fma.rn.f32x2
 * (paired = 1), 2 flops per FMA, best of five timed launches on `stream`
 * (a cudaStream_t, NULL = legacy default).  Synchronous; allocates and frees
 * 4 bytes with the stream-ordered allocator.  MS_ERR_CUDA on failure. */
ms_status ms_peak_fp32(void* stream, int paired, double* tflops);

/* Host-side fault injection: when the environment variable MS_FAULT reads
 * "step:K,code:X" at ms_create (K >= 0, X a non-zero ms_status value), that
 * context's ms_step returns X, without launching, once the context has
 * reached step K, and every later ms_step / ms_sync / ms_diag returns X too
 * (sticky).  Used to test the failure handling of drivers above the library
 * without a device fault.  A malformed MS_FAULT makes ms_create return
 * MS_ERR_ARG. */

/* Step count and physical time of the current state. */
ms_status ms_time(const ms_ctx* ctx, int64_t* step, double* t);

/* Checkpoint / restore of the full state (binary, host buffer). */
size_t ms_checkpoint_bytes(const ms_ctx* ctx);
ms_status ms_checkpoint(ms_ctx* ctx, void* host_buf, size_t bytes);
ms_status ms_restore(ms_ctx* ctx, const void* host_buf, size_t bytes);

/* Moving frame (the SHIFT key of the paper's input files, Sec. 4: a camera
 * that follows the solidification front).  Drops the first `planes` cells
 * along the last axis (z in 3-D, y in 2-D), moves the rest down, fills the far
 * end with pure liquid (the last phase) at chemical potentials mu_fill[K-1]
 * (host array, the original alloy's) and advances the grid's z_origin by
 * `planes`, so the pulled temperature field and the phi-noise counter stay in
 * lab coordinates.  0 <= planes <= extent of the last axis; checkpoints of
 * the adjoint are dropped.  MS_ERR_UNSUPPORTED for a slab of a decomposed
 * domain (MS_BC_HALO along z).  Asynchronous on the context's stream. */
ms_status ms_shift(ms_ctx* ctx, int planes, const double* mu_fill);
/* Highest index along the last axis holding a cell that is not pure liquid
 * (phi of the last phase != 1), -1 if none: the position of the growth front
 * for the moving-frame test.  Synchronises the context's stream. */
ms_status ms_front(ms_ctx* ctx, int* last_plane);

/* Launch shape: tile (index into ms_tile_shapes) and z-chunk (planes marched
 * per CTA, 3-D only; 0 = automatic; values above 64 are clamped to 64). */
ms_status ms_set_launch(ms_ctx* ctx, int tile, int zchunk);
/* Number of tile shapes compiled for this context and their (tx, ty). */
int ms_tile_count(const ms_ctx* ctx);
ms_status ms_tile_shape(const ms_ctx* ctx, int tile, int* tx, int* ty);
/* 1 when tile variant `tile` is a split step (3-D only): a streaming kernel
 * updates the warp rows whose stencil holds one pure phase and lists the
 * others, which a second kernel then updates with the full Sec. 2.1 cell
 * update; results agree with the fused variant of the same tile to FP
 * rounding.  The split variant allocates work lists of 8 bytes per 32-cell
 * row segment (once, through the context's allocator) when first selected.
 * 0 for a fused variant, -1 for a bad index. */
int ms_tile_split(const ms_ctx* ctx, int tile);
/* Current launch: tile index and z-chunk (either pointer may be NULL). */
ms_status ms_get_launch(const ms_ctx* ctx, int* tile, int* zchunk);

/* Autotuner: times every compiled tile shape and a set of z-chunk sizes on
 * the current state (the state is saved and restored), keeps the fastest and,
 * when cache_path is not NULL, records it in that JSON file keyed by device,
 * dim, N, K, dtype and grid, reusing a cached entry when present.
 * best_ms_per_step may be NULL. */
ms_status ms_tune(ms_ctx* ctx, const char* cache_path, int steps_per_trial,
                  double* best_ms_per_step);

/* ---- Discrete adjoint (reverse mode through the explicit steps) ----------
 * Gradients of a loss L on the state after n steps with respect to the
 * initial fields and the parameters theta = (delta_ab for each pair a < b in
 * row-major order, the phase mobility 1/tau, the entries D^a_ij).  The
 * gradient is that of the discrete map the library steps (Eq. phi_eqn and
 * Eq. Mu_explicit_temperature as discretised by ms_step), not of the PDE.
 *
 * ms_enable_checkpoints(ctx, every): from the current step on, ms_step stores
 * a device snapshot of the state every `every` steps (0 turns recording off).
 * Memory: one state per snapshot plus `every` states during ms_grad.
 * Returns MS_ERR_UNSUPPORTED if no adjoint kernel is compiled for the
 * context's (dim, N, K, dtype), with phi noise, the anti-trapping current,
 * grain growth or elasticity on, and for a slab context with halo z faces
 * (the adjoint needs the whole domain).  Resets on ms_set_fields /
 * ms_restore. */
ms_status ms_enable_checkpoints(ms_ctx* ctx, int every);

/* Number of parameters in theta: N(N-1)/2 + 1 + N (K-1)^2. */
int ms_grad_param_count(const ms_ctx* ctx);

/* Reverse pass over the steps run since checkpoints were enabled.
 * dphi_T / dmu_T: dense device arrays dL/dphi and dL/dmu of the current
 * (final) state, layout as ms_set_fields, context dtype; dmu_T may be NULL
 * (zero).  Outputs (each may be NULL): dparams, host array of
 * ms_grad_param_count doubles (dL/dtheta, accumulated in FP64); dphi0 /
 * dmu0, dense device arrays dL/dphi and dL/dmu of the state at the first
 * recorded step.  Synchronous.  Segments between snapshots are recomputed with
 * the forward kernel; per reverse step three adjoint kernels run (per cell,
 * per face, per cell: a gather, no atomics, deterministic).  The current
 * state is left unchanged.  Work buffers (two adjoint states, the per-face
 * records, one segment of `every` states, FP64 partials) are allocated on
 * first use through the context's allocator and kept until ms_destroy.
 * Errors: MS_ERR_STATE without checkpoints or with snapshots missing;
 * MS_ERR_UNSUPPORTED as for ms_enable_checkpoints; MS_ERR_OOM when a work
 * buffer cannot be allocated (nothing is left half-made: the next call
 * allocates what is missing); MS_ERR_CUDA on a failed launch or copy. */
ms_status ms_grad(ms_ctx* ctx, const void* dphi_T, const void* dmu_T, double* dparams,
                  void* dphi0, void* dmu0);

/* ---- Batched form: many independent 2-D simulations, one persistent launch -
 * ms_batch_create: nsims simulations with their own grid (grids[i]) and
 * parameters (params[i]); all share n_phases, n_components and dtype.  This
 * build compiles the batched kernel for 2-D, N = 2, K = 2, FP32 and
 * time-independent temperature (G V = 0); other combinations return
 * MS_ERR_UNSUPPORTED.  Each simulation keeps its own ping-pong state and
 * its own TMA descriptor in device memory.
 * ms_batch_step(b, n): advances every simulation n steps in ONE cooperative,
 * persistent kernel launch that walks a (simulation, tile) work list with a
 * bounded-spin grid barrier between steps; the launch is captured once into a
 * CUDA graph per (n, buffer parity) and replayed.  Asynchronous; a barrier
 * timeout is reported by ms_batch_sync as MS_ERR_TIMEOUT.
 * Field I/O per simulation as in ms_set_fields / ms_get_fields (synchronous
 * for host buffers). */
ms_status ms_batch_create(int nsims, const ms_grid* grids, int n_phases, int n_components,
                          const ms_params* params, void* stream, const ms_allocator* alloc,
                          ms_batch** out);
void ms_batch_destroy(ms_batch* b);
const char* ms_batch_last_error(const ms_batch* b);
ms_status ms_batch_set_fields(ms_batch* b, int sim, const void* phi, const void* mu, int on_device);
ms_status ms_batch_get_fields(ms_batch* b, int sim, void* phi, void* mu, int on_device);
ms_status ms_batch_step(ms_batch* b, int64_t n);
ms_status ms_batch_sync(ms_batch* b);
int64_t ms_batch_cells(const ms_batch* b);   /* total cells over all simulations */
/* Tile height of the batched work list: the persistent kernel is compiled for
 * 32 x 4, 32 x 8 (the default) and 32 x 16 tiles; a change rebuilds the work
 * list and the tensor maps (synchronous) and recaptures the graph at the next
 * ms_batch_step.  MS_ERR_ARG for another height. */
ms_status ms_batch_set_tile(ms_batch* b, int tile_height);
int ms_batch_tile(const ms_batch* b);        /* current tile height, 0 for NULL */
/* Autotuner of the batched form: times steps_per_trial steps (after one
 * warm-up launch of the same length) with every compiled tile height on the
 * current states, restores the states (a device copy of all of them is held
 * during the call) and keeps the fastest height; best_ms_per_step (may be
 * NULL) receives its time per step.  Synchronous. */
ms_status ms_batch_tune(ms_batch* b, int steps_per_trial, double* best_ms_per_step);

/* ---- Slab decomposition along z (3-D) ---------------------------------------
 * A domain split into contexts that each own a contiguous range of z-planes
 * (grid.bc[2] = MS_BC_HALO, grid.z_origin = the slab's first global plane, so
 * the temperature field stays global) advances exactly like the whole domain
 * when, after every step (and once after ms_set_fields), each internal cut is
 * exchanged and each outer no-flux face is mirrored.  The exchange copies one
 * padded z-plane of every field (and of the bulk codes) in each direction:
 * the one exchange step of the explicit scheme (stencil radius 1).
 * ms_halo_exchange(lower, upper): lower's top plane -> upper's bottom ghost,
 *   upper's bottom plane -> lower's top ghost.  Same nx, ny, N, K, dtype and
 *   the same stream are required (MS_ERR_ARG otherwise); enqueued on it.
 *   For a periodic domain, also exchange (last, first).
 * ms_halo_mirror(ctx, face): face 0 = bottom, 1 = top; no-flux ghost plane
 *   (copy of the adjacent interior plane) for an outer face of a slab. */
ms_status ms_halo_exchange(ms_ctx* lower, ms_ctx* upper);
ms_status ms_halo_mirror(ms_ctx* ctx, int face);

/* The same exchange between processes (slabs held by different ranks: the
 * domain decomposition with buffer layers of the paper's Sec. "CPU (MPI)
 * implementation" and the GPU subdomains of Sec. "CUDA implementation"):
 * a boundary plane travels through a flat device buffer that the caller
 * moves between ranks (e.g. with torch.distributed or NCCL).
 * ms_halo_plane_bytes: bytes of one packed plane, 0 for a 2-D context:
 *   one padded z-plane of every field ([field][nyp][pitch] elements in the
 *   context dtype, x/y ghost cells included) followed by the plane's
 *   segment codes ([ny][segs] bytes).
 * ms_halo_pack(ctx, face, dst): face 0 = the bottom interior plane (z = 0),
 *   face 1 = the top interior plane (z = nz - 1) -> dst (device, at least
 *   ms_halo_plane_bytes).
 * ms_halo_unpack(ctx, face, src): a packed plane from the neighbour ->
 *   the ghost plane on that face (0 = below z = 0, 1 = above z = nz - 1).
 * After every step (and once after ms_set_fields), each rank packs both
 * faces, sends face 1 up and face 0 down, and unpacks what it receives into
 * the matching ghost planes (outer no-flux faces: ms_halo_mirror).  Both are
 * asynchronous on the context's stream (synchronise it before handing dst to
 * another stream or rank).  MS_ERR_ARG for a context without MS_BC_HALO z
 * faces. */
size_t ms_halo_plane_bytes(const ms_ctx* ctx);
ms_status ms_halo_pack(ms_ctx* ctx, int face, void* dst);
ms_status ms_halo_unpack(ms_ctx* ctx, int face, const void* src);

/* ---- Sparse grain growth: many grains, few per cell ------------------------
 * Isotropic grain growth (GRAINGROWTH = 1, Sec. 4 "Grain-growth": the phi
 * equation of Sec. 2.1 without the chemical driving force) with up to 64
 * grains, every cell storing only the grains non-zero there (at most 8: a
 * grain index and a value each).  The Lagrange multiplier is taken over the
 * locally active grains -- those non-zero at the cell or at one of its face
 * neighbours: the projection onto the simplex runs over them alone and every
 * other grain stays 0 -- so a grain appears only next to where it is.  The
 * obstacle potential (Eq. Obstacle) with a uniform triple term Gamma_abc
 * (gamma3, the same value for every triple of distinct grains; a value above
 * 96 gamma / pi^2 keeps third grains out of two-grain boundaries) and
 * isotropic pairs (delta = 0); no mu field.
 * ms_ggs_create(grid, n_grains, params, stream, alloc, out): params as for
 *   ms_create (dtype, eps, tau, dt, gamma [N][N], gamma3 [N][N][N] or NULL;
 *   potential MS_POT_OBSTACLE; noise, anti-trapping, elasticity off); the
 *   whole domain (no MS_BC_HALO).  dt is checked against the explicit bound
 *   (dx^2 / 2 dim) tau / gamma_max (MS_ERR_DT_UNSTABLE).  MS_ERR_ARG /
 *   MS_ERR_UNSUPPORTED for other settings.
 * ms_ggs_set_fields(ctx, phi, on_device): phi dense [N][z][y][x] in the
 *   context dtype; a cell with more than 8 non-zero grains, or a negative or
 *   non-finite value, gives MS_ERR_BOUNDS.  Resets the step counter.
 * ms_ggs_get_fields(ctx, phi, on_device): the dense fields (zeros where a
 *   grain is absent); synchronous.
 * ms_ggs_step(ctx, n): n steps (two launches each: the cells whose 7-point
 *   stencil is one grain keep it, the others are listed and updated).
 *   Asynchronous on the context's stream.
 * ms_ggs_sync(ctx): waits; MS_ERR_BOUNDS (sticky) when a step needed more than
 *   8 grains in a cell or in a cell's stencil.
 * ms_ggs_stats(ctx, listed_cells, step): cells updated by the last step's
 *   list and the step count (synchronises). */
typedef struct ms_ggs ms_ggs;
ms_status ms_ggs_create(const ms_grid* grid, int n_grains, const ms_params* params, void* stream,
                        const ms_allocator* alloc, ms_ggs** out);
void ms_ggs_destroy(ms_ggs* ctx);
const char* ms_ggs_last_error(const ms_ggs* ctx);
ms_status ms_ggs_set_fields(ms_ggs* ctx, const void* phi, int on_device);
ms_status ms_ggs_get_fields(ms_ggs* ctx, void* phi, int on_device);
ms_status ms_ggs_step(ms_ggs* ctx, int64_t n);
ms_status ms_ggs_sync(ms_ggs* ctx);
ms_status ms_ggs_stats(ms_ggs* ctx, int64_t* listed_cells, int64_t* step);

/* Allocation-free diagnostics (the paper has no counterpart; this is a
 * library service).  For callers that cannot allocate device memory while
 * they run -- a host application that gives this library a fixed memory
 * budget, code being recorded into a CUDA graph by stream capture (where a
 * cudaMalloc would break the capture), or a latency-bound loop that must not
 * stall on the allocator.  It computes the same quantities as ms_diag
 * (out[0..K-2] solute masses, out[K-1] max |sum phi - 1|, out[K] min phi,
 * out[K+1] max phi, out[K+2] non-finite count, out[K+3] mu-diffusion number)
 * for a state the caller holds: phi_dev / mu_dev are dense device arrays
 * [field][z][y][x] in params->dtype, t the physical time of that state, and
 * out_dev a device buffer of at least K+4 doubles written on `stream`
 * (asynchronously; synchronise the stream before reading it).
 *   - No device memory is allocated or freed: the per-block reduction scratch
 *     is a fixed array in the library's device image (512 KiB per GPU that
 *     loads the library, held until the process exits).
 *   - Size limit: grids of at most 268,435,456 cells (8192 blocks of 32,768
 *     cells); larger grids return MS_ERR_BOUNDS with a message.
 *   - The first call on each device resolves the scratch array's device
 *     address (cudaGetSymbolAddress) with that device current; make that
 *     first call before starting any stream capture on that device.
 *   - All calls share the one scratch array, so calls whose kernels overlap on
 *     the GPU (different streams without ordering) race and may return wrong
 *     values; order them on one stream or with events.
 *   - Errors: MS_ERR_ARG for bad inputs, MS_ERR_UNSUPPORTED for a
 *     (dim, N, K) without compiled diagnostics, MS_ERR_BOUNDS as above,
 *     MS_ERR_CUDA for a failed launch; text via ms_last_error(NULL). */
ms_status ms_diag_noalloc(const ms_grid* grid, int n_phases, int n_components,
                          const ms_params* params, double t, const void* phi_dev,
                          const void* mu_dev, double* out_dev, void* stream);
#define MS_DIAG_NOALLOC_LEN(K) ((K) + 4)

#ifdef __cplusplus
}
#endif
#endif /* MICROSIM_GB_H */
