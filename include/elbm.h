/*
 * elbm.h - C ABI of the GB300 (sm_103a) two-population compressible lattice
 * Boltzmann library (Saadat, Hosseini, Dorschner & Karlin, arXiv:2102.09512).
 *
 * One time step updates both populations at every node (Eqs. fLBGK, gLBGK):
 *   f_i(x + c_i, t + 1) = f_i + omega (f_i^ex - f_i)
 *   g_i(x + c_i, t + 1) = g_i + omega_1 (g_i^eq - g_i) + (omega - omega_1)(g_i^eq - g_i^*)
 * with the extended equilibrium f^ex (Eqs. extf, Pa_star), the operator
 * product-form energy equilibrium g^eq (Eq. geq_i), the quasi-equilibrium g*
 * (Eqs. gstar, qstar1), omega and omega_1 from mu and Pr (Eqs. mu, Pr), T from the
 * total energy of an ideal gas with constant Cv = 1/(gamma - 1) (Eqs. U, E; R = 1),
 * and the derivative of the anomaly Q~_aaa (Eq. anomalya) by first-order upwind
 * differences (Sec. III.A).  Lattice units: dx = dt = 1.
 *
 * Conventions
 *  - Node index n = x + nx*(y + ny*z).  Host and device field arrays are FP64:
 *    rho[N], T[N], u[D*N] component-major (u_x block, then u_y, then u_z).
 *  - Memory: the caller owns every device buffer (two population stores and one
 *    auxiliary buffer, sizes from elbm_bytes_required) and the stream; the library
 *    owns only the handle.  Population layout: Q planes of N elements, element
 *    [i*N + n] holding the pair (f_i, g_i) of direction i = (c_x+1) + 3(c_y+1) +
 *    9(c_z+1) at node n (both are pulled from the same source node, so one access
 *    moves both).  Device pointers must be 256-byte aligned.
 *    The store holds the post-collision populations of the current time level
 *    (streaming is a pull at the start of the next step); their moments rho,
 *    rho u, rho E equal those of the post-stream state because the collision
 *    conserves them.
 *  - Calls are asynchronous on the bound stream unless stated; functions that
 *    return host data synchronise the stream.
 *  - Errors: every function returns an elbm_status (0 = ELBM_OK).  Argument errors
 *    are reported synchronously.  Conditions found on the device (non-finite
 *    moments, rho <= 0 or T <= 0) are latched in the auxiliary buffer and reported
 *    by the next synchronising call as ELBM_ERR_NONPHYSICAL; a bounded device wait
 *    that gave up (ELBM_KERNEL_FUSED_TMA) is reported as ELBM_ERR_TIMEOUT.
 *  - A handle is not thread-safe.
 */
#ifndef ELBM_H
#define ELBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ELBM_OK = 0,
    ELBM_ERR_ARG = -1,          /* invalid argument or unbound handle            */
    ELBM_ERR_UNSUPPORTED = -2,  /* valid but not implemented combination        */
    ELBM_ERR_CUDA = -3,         /* a CUDA runtime call failed                     */
    ELBM_ERR_NONPHYSICAL = -4,  /* device saw a non-finite value, rho<=0 or T<=0 */
    ELBM_ERR_TIMEOUT = -5       /* a bounded device wait gave up                  */
} elbm_status;

typedef enum { ELBM_D2Q9 = 9, ELBM_D3Q27 = 27 } elbm_lattice;

/* Per face -x,+x,-y,+y,-z,+z.  An axis is periodic on both faces or on neither.
 * Zero-gradient: the ghost node holds a copy of the adjacent interior node (its
 * post-collision populations and its Q~); the paper states no boundary type.
 * Fixed state (a supersonic inflow, as upstream of the shock in Sec. III.C): the
 * ghost holds the equilibria f^eq, g^eq of the uniform state fix_rho, fix_u, fix_T
 * of elbm_params (their own post-collision values) and that state's Q~; D2Q9 only
 * (ELBM_ERR_UNSUPPORTED for D3Q27). */
typedef enum { ELBM_BC_PERIODIC = 0, ELBM_BC_ZEROGRAD = 1, ELBM_BC_FIXED = 2 } elbm_bc;

/* Population storage.  F64 and F32 store the populations; F16DEV and BF16DEV store
 * their deviation from the rest state f^eq(rho_ref, 0, T_ref), g^eq(rho_ref, 0, T_ref)
 * rounded to nearest even, with FP32 arithmetic. */
typedef enum { ELBM_F64 = 0, ELBM_F32 = 1, ELBM_F16DEV = 2, ELBM_BF16DEV = 3 } elbm_store;

/* Caloric equation of state of the ideal gas (Eqs. U, E; R = 1, reference temperature
 * 0): constant Cv = 1/(gamma - 1), or Cv(T) = cv[0] + cv[1] T + cv[2] T^2 + cv[3] T^3
 * with U(T) = int_0^T Cv dT (gamma then unused; cv[0] > 0 and Cv must stay positive
 * over the run's temperatures).  T is recovered from U by Newton's method. */
typedef enum { ELBM_EOS_GAMMA = 0, ELBM_EOS_CV_POLY = 1 } elbm_eos;

/* Spatial derivative of Q~_aaa: first-order upwind (the paper's choice, Sec. III.A)
 * or second-order central (its comparison variant). */
typedef enum { ELBM_DERIV_UPWIND = 0, ELBM_DERIV_CENTRAL = 1 } elbm_deriv;

/* Kernel schedule of one step. */
typedef enum {
    ELBM_KERNEL_FUSED = 0,        /* one kernel: halo-recomputed moments + collide + stream;
                                     D3Q27 FP32/FP16/BF16 prefetch each plane into shared
                                     memory (cp.async), FP64 uses the re-read form; D2Q9
                                     marches strips of 128 nodes along y with the next rows
                                     prefetched into shared memory (cp.async), or runs one
                                     32 x 8 tile per CTA on grids too small for the march
                                     to fill the device (see elbm_set_tile_z) */
    ELBM_KERNEL_TWOPASS = 1,      /* moment/Q~ pass into the aux buffer, then collide+stream */
    ELBM_KERNEL_FUSED_REREAD = 2, /* one kernel, D3Q27 plane gathered twice (second from L2);
                                     D2Q9: one 32 x 8 tile per CTA, no march */
    ELBM_KERNEL_FUSED_TMA = 3     /* one kernel, D3Q27 FP32/FP16/BF16: each plane is staged in
                                     shared memory by the tensor-copy engine (TMA), one box per
                                     direction, where the boxes of a tile lie inside the grid,
                                     and by per-pair cp.async copies at the x and y faces; a
                                     plane's arrival is counted on an mbarrier.  Needs nx a
                                     multiple of 2 (FP32) or 4 (FP16/BF16), otherwise
                                     elbm_set_kernel returns ELBM_ERR_UNSUPPORTED (also
                                     returned by elbm_step if the driver refused the tensor
                                     maps at elbm_bind).  Its waits are bounded (about 1 s):
                                     one that gives up is reported as ELBM_ERR_TIMEOUT by the
                                     next synchronising call */
} elbm_kernel;

/* Storage of the populations.  Ping-pong: two stores, a step reads one and writes the
 * other (every schedule).  AA: one store updated in place, its layout alternating with the
 * step parity (after an even number of steps the pairs of a node sit at the node with each
 * direction in the opposite direction's plane; after an odd number, each pair sits at the
 * node it streams to next), on the two-pass schedule: the first pass writes the Q~ field,
 * the second reads and writes exactly the slots each node read, so no two threads touch one
 * slot.  Half the population memory (D3Q27 FP32 at 1024^3: 232 GB instead of 464 GB), 1.5x
 * the bytes per update of the fused schedule.  Periodic grids only (a zero-gradient or fixed
 * face makes two nodes read one slot that one of them writes). */
typedef enum { ELBM_LAYOUT_PINGPONG = 0, ELBM_LAYOUT_AA = 1 } elbm_layout;

typedef struct {
    int lattice;         /* ELBM_D2Q9 or ELBM_D3Q27                                  */
    int nx, ny, nz;      /* grid; nz must be 1 for D2Q9                               */
    double gamma;        /* adiabatic exponent (Eq. gamma), > 1                        */
    double Pr;           /* Prandtl number (Eq. Pr), > 0                               */
    double mu0;          /* dynamic viscosity at T0 (Eq. mu), > 0                      */
    double T0;           /* reference temperature of the power law, > 0               */
    double mu_exp;       /* mu = mu0 (T/T0)^mu_exp; 0 = constant (Sec. III.D uses 0.76) */
    int bc[6];           /* elbm_bc per face                                          */
    int store;           /* elbm_store                                                */
    int deriv;           /* elbm_deriv                                                */
    double rho_ref;      /* rest state of the deviation stores (ignored for F64/F32)  */
    double T_ref;
    double fix_rho;      /* state of the ELBM_BC_FIXED faces (ignored without one):    */
    double fix_u[3];     /*   density > 0, velocity, temperature > 0                   */
    double fix_T;
    int eos;             /* elbm_eos                                                  */
    double cv[4];        /* Cv(T) coefficients for ELBM_EOS_CV_POLY                    */
} elbm_params;

typedef struct elbm_handle elbm_handle;

/* Validates the parameters and creates a handle.  Host-only, no CUDA call. */
int elbm_create(const elbm_params *params, elbm_handle **out);

/* Selects the population storage (elbm_layout) before elbm_bind; ELBM_LAYOUT_AA needs a
 * grid periodic on every axis (otherwise ELBM_ERR_UNSUPPORTED) and selects the two-pass
 * schedule (elbm_set_kernel then accepts ELBM_KERNEL_TWOPASS only).  Host field transfers of
 * an AA handle are staged in chunks of 2^25 nodes, so its auxiliary buffer stays small.
 * Host-only. */
int elbm_set_layout(elbm_handle *h, int layout);

/* Bytes of each population store (one store for ELBM_LAYOUT_AA, two otherwise) and of the
 * auxiliary buffer (status word, reduction partials, the Q~ field of the two-pass schedule
 * and a staging area for host field transfers). */
int elbm_bytes_required(const elbm_handle *h, size_t *pop_bytes, size_t *aux_bytes);

/* Binds caller-owned device buffers and a stream (cudaStream_t, may be NULL for
 * the legacy default stream).  pop_a and pop_b are the two ping-pong stores; the
 * state lives in pop_a after elbm_set_fields*.  With ELBM_LAYOUT_AA, pop_a is the single
 * store and pop_b is NULL (or pop_a).  Clears the status word. */
int elbm_bind(elbm_handle *h, void *pop_a, void *pop_b, void *aux, void *stream);

/* Initial state f = f^eq(rho,u,T), g = g^eq(rho,u,T) (no non-equilibrium part).
 * _device: FP64 device arrays; plain: host arrays, synchronising.  Host arrays in
 * page-locked memory the device maps (cudaHostAlloc, cudaMallocHost, cudaHostRegister),
 * each inside one allocation, are read by the initialisation kernel directly over the
 * host link; other host memory is copied through the aux staging area.  The results
 * are the same either way. */
int elbm_set_fields(elbm_handle *h, const double *rho, const double *u, const double *T);
int elbm_set_fields_device(elbm_handle *h, const double *rho, const double *u, const double *T);

/* Advances nsteps time steps with the selected kernel schedule (asynchronous). */
int elbm_step(elbm_handle *h, int nsteps);

/* Steps replayed from CUDA graphs (for grids small enough that launching is what a step
 * costs): with steps_per_graph = G > 0, elbm_step runs whole groups of G steps as one
 * replay each of a graph captured on first use (one per starting store, or AA layout
 * parity) and the remainder as single steps.  The replays launch the same kernels with
 * the same arguments as single steps, so the results are the same.  The graphs hold the
 * bound buffers, the kernel schedule and the kernel parameters; elbm_bind, elbm_set_kernel,
 * elbm_set_tile_z and elbm_inject_wait_timeout drop them.  G = 0 (the default) turns
 * replays off; G must be even (a replay ends at the parity it began) and at most 1024,
 * else ELBM_ERR_ARG.  Not for use while the caller captures the handle's stream itself. */
int elbm_set_step_graph(elbm_handle *h, int steps_per_graph);

/* rho, u, T of the current state (Eqs. density, momentum, energy, E).
 * Plain: host arrays, synchronises and returns the latched device status (page-locked
 * mapped host arrays are written by the field kernel directly, as for elbm_set_fields).
 * _device: FP64 device arrays, asynchronous. */
int elbm_get_fields(elbm_handle *h, double *rho, double *u, double *T);
int elbm_get_fields_device(elbm_handle *h, double *rho, double *u, double *T);

/* Totals {sum rho, sum rho u_x, sum rho u_y, sum rho u_z, sum rho E} of the current
 * state, FP64 with compensated summation (Eqs. density, momentum, energy).
 * Synchronises. */
int elbm_conservation(elbm_handle *h, double out[5]);

/* The same totals accumulated inside the last step's kernel from the populations
 * it pulled (the state that step produced; the collision conserves the totals).
 * FP64 stores: FP64 throughout; other stores: FP32 sums per thread (over the planes a
 * thread updates) and per warp, FP64 across warps and CTAs (relative rounding of order
 * 1e-7, below that of the FP32 node values).  Synchronises. */
int elbm_step_totals(elbm_handle *h, double out[5]);

/* The same totals without synchronising: enqueues on the handle's stream the reduction
 * of the last step's per-CTA sums and the copy of the five totals into out, and
 * returns.  out must stay valid until the stream has passed that point (an event
 * recorded after the call, cudaStreamSynchronize, or any synchronising call of this
 * library); with out in page-locked host memory the copy is asynchronous too, so the
 * caller can enqueue the next steps before reading the totals of this one.  The latched
 * status is not read (the next synchronising call reports it).  ELBM_ERR_ARG before the
 * first step. */
int elbm_step_totals_async(elbm_handle *h, double out[5]);

/* Turbulence statistics of the current state (paper Sec. III.D), volume averages
 * over all nodes, FP64: out = {<rho>, rho_rms, K = <rho u.u>/2, u_rms = sqrt(<u.u>/D),
 * theta_rms = sqrt(<(div u)^2>), <T>, T_rms, <(d u_x/d x)^2>,
 * omega_rms = sqrt(<|omega|^2>), enstrophy = <|omega|^2>/2,
 * dissipation = <mu(T) |omega|^2>, lambda = sqrt(<u_x^2>/<(d u_x/d x)^2>),
 * Re_lambda = <rho> u_rms lambda / mu0} with omega = curl u; derivatives by
 * second-order central differences (ghosts from the boundary map).  out holds 13
 * doubles (caller-owned).  Synchronises. */
int elbm_turbulence_stats(elbm_handle *h, double out[13]);

/* Selects the kernel schedule (elbm_kernel).  Results agree to rounding. */
int elbm_set_kernel(elbm_handle *h, int kernel);

/* Length of the segment each CTA of the fused kernel marches over: z planes for
 * D3Q27, rows (y) for D2Q9.  Chosen at elbm_create for the current device (the
 * length that best fills the last wave of CTAs, each segment costing about two
 * planes of prologue); a tuning knob, results agree to rounding.  D2Q9 grids with
 * fewer 128-node strips x row segments than the device has SMs run the fused schedule
 * as one 32 x 8 tile per CTA instead of the march; setting a segment length here
 * selects the march for any grid. */
int elbm_set_tile_z(elbm_handle *h, int tz);

/* Raw copy of the current population store (pop_bytes) to or from host memory,
 * for checkpoint and restart.  Synchronises.  An AA store is copied in its current
 * layout: restore it into a handle at the same step parity (elbm_steps_done). */
int elbm_get_populations(elbm_handle *h, void *host_dst);
int elbm_set_populations(elbm_handle *h, const void *host_src);

/* Synchronises the stream and returns the latched device status (and clears it). */
int elbm_sync(elbm_handle *h);

/* Fault injection for testing the failure path of ELBM_KERNEL_FUSED_TMA: with on = 1,
 * every plane a tile requests by tensor copies announces 16 bytes more than the copies
 * deliver, so the tile's bounded wait (about one second) runs out; the kernel then
 * waits, again bounded, for its copies, ends the tile and latches the timeout, which the
 * next synchronising call returns as ELBM_ERR_TIMEOUT.  The step's results are invalid;
 * the handle and the CUDA context stay usable (set the fields again).  on = 0 restores
 * normal operation.  No effect on the other schedules. */
int elbm_inject_wait_timeout(elbm_handle *h, int on);

/* Number of time steps taken since the last elbm_set_fields*. */
long long elbm_steps_done(const elbm_handle *h);

/* Number of kernel launches this handle has issued (for launch accounting). */
long long elbm_launch_count(const elbm_handle *h);

/* Velocity c_i = (c[0], c[1], c[2]) of direction i of a lattice (Eq. d3q27vel). */
int elbm_velocity(int lattice, int i, int c[3]);

/* One time step, src -> dst, of the two-pass schedule, for callers that cannot
 * allocate device memory (for example a solver embedded in an application that owns
 * the whole device memory pool and lends the library only the populations it
 * updates).  No handle and no auxiliary buffer: the scratch this step needs (the Q~
 * field, the per-CTA partials and the status word) lives in a fixed static device
 * array of 16 MiB that every GPU loading the library holds until the process exits.
 * The paper has no counterpart; this is an interface choice of the library.
 *   params  problem statement, validated as by elbm_create;
 *   src     current population store (device, pop_bytes, 256-byte aligned, read);
 *   dst     next population store (device, pop_bytes, 256-byte aligned, written);
 *   stream  cudaStream_t (NULL: legacy default stream); the call is asynchronous.
 * Limits: the Q~ field and partials must fit the array: about 1.37 M nodes for
 * D3Q27 with FP32/FP16/BF16 stores, 0.69 M for FP64, 2.05 M for D2Q9 FP32; larger
 * grids return ELBM_ERR_UNSUPPORTED before anything is launched.
 * The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.  The
 * address belongs to the device's context: after a cudaDeviceReset the next call looks
 * it up again, so make the first call after a reset before any capture as well.
 * Calls no cudaMalloc, cudaFree or other allocating routine.  All calls share the
 * array, so calls whose kernels overlap on the GPU (different streams, or several
 * host threads) race on it; serialise them.  The status word is cleared by each
 * call and device-detected non-physical states are not reported here (read them
 * through the handle API, e.g. elbm_conservation on a bound handle). */
int elbm_step_noalloc(const elbm_params *params, const void *src, void *dst, void *stream);

/* Frees the handle (not the caller's buffers). */
int elbm_destroy(elbm_handle *h);

/* ---------------------------------------------------------------------------
 * Ensembles: n independent D2Q9 lattices of uneven sizes (the paper's 2D cases run
 * side by side, e.g. a sweep of Mach numbers and grid sizes), all with the same
 * store kind, kept back to back in one pair of population stores.  Each instance
 * follows exactly the single-lattice update above.
 * ------------------------------------------------------------------------- */
typedef struct elbm_ensemble elbm_ensemble;

typedef enum {
    ELBM_ENSEMBLE_PERSISTENT = 0,   /* one launch per step over the tiles of all instances */
    ELBM_ENSEMBLE_PER_INSTANCE = 1  /* one fused launch per instance per step               */
} elbm_ensemble_mode;

/* Validates params[0..n-1] (each as for elbm_create; D2Q9 only, one store kind,
 * 1 <= n <= 1024) and creates the ensemble.  Host-only. */
int elbm_ensemble_create(const elbm_params *params, int n, elbm_ensemble **out);
int elbm_ensemble_bytes_required(const elbm_ensemble *e, size_t *pop_bytes, size_t *aux_bytes);
/* Binds caller-owned device buffers (256-byte aligned) and a stream; copies the
 * instance tables into the auxiliary buffer (synchronising). */
int elbm_ensemble_bind(elbm_ensemble *e, void *pop_a, void *pop_b, void *aux, void *stream);
/* Initial state of instance k from host FP64 fields (layout as elbm_set_fields). */
int elbm_ensemble_set_fields(elbm_ensemble *e, int k, const double *rho, const double *u, const double *T);
int elbm_ensemble_get_fields(elbm_ensemble *e, int k, double *rho, double *u, double *T);
/* Schedule: persistent (optionally replayed from a CUDA graph) or one launch per
 * instance.  Results are identical. */
int elbm_ensemble_set_mode(elbm_ensemble *e, int mode, int use_graph);
/* Persistent schedule: the work unit and resident CTAs per SM (the grid is that times
 * the SM count, capped by the unit count).  tile_y = 4, 8 or 16: one tile of 32 x tile_y
 * nodes per unit; tile_y = 32, 64 or 128: a strip of 128 nodes of an instance marched
 * along y over a segment of tile_y rows (next rows prefetched into shared memory). */
int elbm_ensemble_set_schedule(elbm_ensemble *e, int tile_y, int ctas_per_sm);
int elbm_ensemble_get_schedule(const elbm_ensemble *e, int *tile_y, int *ctas_per_sm, int *grid);
/* Autotuner: times every (work unit, CTAs per SM) the hardware can hold over
 * trial_steps steps each and keeps the fastest; with use_cache, a schedule tuned
 * before for the same store kind and size class (log2 of the node count) is reused.
 * The candidates write only the spare store, so the state is unchanged. */
int elbm_ensemble_tune(elbm_ensemble *e, int trial_steps, int use_cache);
/* Advances every instance nsteps steps (asynchronous).  With the persistent schedule and
 * graphs on, each group of 8 steps replays one CUDA graph of 8 launches (built on first
 * use) and the remaining steps one graph of one launch each. */
int elbm_ensemble_step(elbm_ensemble *e, int nsteps);
/* Synchronises and returns (and clears) the latched device status. */
int elbm_ensemble_sync(elbm_ensemble *e);
long long elbm_ensemble_launch_count(const elbm_ensemble *e);
long long elbm_ensemble_nodes(const elbm_ensemble *e);
int elbm_ensemble_destroy(elbm_ensemble *e);

/* Static string for a status code. */
const char *elbm_status_str(int code);

#ifdef __cplusplus
}
#endif

#endif /* ELBM_H */
