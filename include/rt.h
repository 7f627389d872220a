/*
 * rt.h -- C ABI of the GB300 radiation-transfer step library.
 *
 * The library advances the frequency-integrated specific intensity
 * I(x, n_m) of Jiang, Stone & Davis (2014, arXiv:1403.6126) by one time step
 * on a Cartesian grid, on one GPU:
 *   transport   (sec. 4.2, eqs. decomposeI and transporttwoterms, the alpha
 *                factor, van Leer faces as eq. 4 of Stone & Mihalas 1992)
 *   velocity    (sec. 4.5, the half-step estimate v~)
 *   absorption  (sec. 4.3, eq. absorptionmatrix, implicit with the T^4 gas
 *                energy exchange)
 *   scattering  (sec. 4.4, the matrix M_s, implicit)
 *   quadrature  (sec. 3: E_r = 4 pi sum W I, F_r = 4 pi sum W n I,
 *                P_r = 4 pi sum W n n I) and the gas source terms
 *                (eqs. momentumchange and kinetichange).
 * All quantities are dimensionless as in sec. 2 (eq. RTequation): Crat is
 * the speed of light, Prat the radiation-to-gas pressure ratio.  The MHD
 * update (Steps 6-7 of sec. 4.1) is the caller's: density, temperature and
 * velocity enter as given fields.
 *
 * Conventions for every call:
 *  - Arrays are plain pointers.  Cell arrays have N = n[0]*n[1]*n[2] entries,
 *    x fastest: cell (i, j, k) is at i + n[0]*(j + n[1]*k).  Vector fields
 *    are component-major: v[d*N + c].  The pressure tensor is P[q*N + c]
 *    with q = xx, yy, zz, xy, xz, yz.  Intensities are angle-major:
 *    I[m*N + c], angles in the caller's order.
 *  - Host pointers unless rt_options.device_ptrs is set, in which case every
 *    array argument of rt_set_material / rt_set_intensity / rt_moments /
 *    rt_sources / rt_get_intensity is a device pointer (doubles) valid on
 *    the context's device; the call reads or writes it on the context's
 *    stream and returns when the work is queued (stream-ordered).
 *  - The caller owns every array it passes; the library copies what it keeps.
 *    The library owns contexts, servers and all device state they hold.
 *  - Every call returns an rt_status and never aborts the process.  On an
 *    error the context is left as it was before the call (except RT_E_CUDA,
 *    after which the context should be destroyed) and rt_last_error() gives
 *    a message for the calling thread.
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RT_OK = 0,
  RT_PENDING = 1,       /* rt_poll: the solve has not finished yet           */
  RT_E_INVALID = -1,    /* bad argument (size, NULL, non-unit n, sum W != 1) */
  RT_E_NOMEM = -2,      /* device or host allocation failed                  */
  RT_E_BUDGET = -3,     /* request larger than the server's HBM budget       */
  RT_E_CUDA = -4,       /* a CUDA call failed                                */
  RT_E_NONFINITE = -5,  /* non-finite input, or the T^4 Newton did not converge */
  RT_E_TIMEOUT = -6,    /* rt_server_wait timed out                          */
  RT_E_STATE = -7       /* call out of order (e.g. rt_step before material)  */
} rt_status;

/* Boundary kinds (the setups of sec. 5): PERIODIC wraps; VACUUM copies
 * outgoing rays and zeroes incoming ones (sec. 5.3 top); COPY copies all
 * rays from the last active cell (sec. 5.3 bottom, sec. 5.8 right side);
 * INFLOW copies outgoing rays and sets incoming ones to per-angle values
 * given by rt_set_inflow (sec. 5.8 beams). */
enum { RT_BC_PERIODIC = 0, RT_BC_VACUUM = 1, RT_BC_COPY = 2, RT_BC_INFLOW = 3 };

/* Storage precision of the intensity.  RT_FP64: everything in double.
 * RT_FP32: intensities, transport and angle sums in float (compensated
 * sums), the T^4 solve finished in double, T and the gas energy source in
 * double.  RT_BF16: the RT_FP32 arithmetic with each intensity stored in
 * 16 bits as its deviation from the cell's mean intensity, delta_m =
 * I_m / J - 1 with J = E_r / (4 pi) (bf16 keeps 8 significant bits, so
 * storing I_m costs a relative error up to 2^-8 |delta_m|); an extra float
 * M x N scratch holds the implicit right-hand sides; one tile shape per
 * dimension; not for batches or the server.  An experiment: the paper
 * stores double intensities. */
enum { RT_FP64 = 0, RT_FP32 = 1, RT_BF16 = 2 };

/* Angle-set generators for rt_angle_set. */
enum { RT_ANGLES_LEVEL_SYMMETRIC = 0,  /* S_N, order N in {2,4,6,8}: N(N+2) angles */
       RT_ANGLES_GAUSS_LEGENDRE = 1,   /* 1-D slab, order = number of angles (1..64) */
       RT_ANGLES_PAPER_S4 = 2 };       /* 24 angles, mu_1 = 1/3 (sec. 5.2)   */

typedef struct rt_ctx rt_ctx;

/* Grid.  dim = 1, 2 or 3 active axes (x, then y, then z); n[d] cells on
 * axis d (1 on inactive axes); the domain is [lo[d], hi[d]] so the cell
 * size is (hi - lo) / n.  bc[d][0] / bc[d][1] are the lower / upper faces
 * of active axes (ignored on inactive ones). */
typedef struct {
  int dim;
  int n[3];
  double lo[3], hi[3];
  int bc[3][2];
} rt_grid;

/* Angle set (sec. 3): m unit vectors n[3*l + d] and weights w[l].  The
 * weights must sum to 1 (J = sum W I is the mean intensity, E_r = 4 pi J)
 * and each |n| must be 1, both to 1e-12; host memory, copied by rt_create. */
typedef struct {
  int m;
  const double *n;
  const double *w;
} rt_angles;

/* Options.  Defaults (rt_options_default): RT_FP32, cfl 0.4 (Step 1 of
 * sec. 4.1), gamma 5/3, r_ideal 1, hold_T 0, estimate_v 1, device_ptrs 0,
 * stream NULL (the legacy default stream), newton_max_it 60, newton_rtol
 * 1e-13.
 *
 * The Newton iteration on the gas temperature (Step 4, sec. 4.3: the paper
 * solves eq. absorptionmatrix by Newton-Raphson and notes that it converges
 * in a few iterations) starts from T^n and stops once a step changes T by
 * at most newton_rtol * T, after one more step; a cell that needs more than
 * newton_max_it steps, or whose iterate leaves T > 0, counts as a failure
 * (rt_sync then returns RT_E_NONFINITE).  newton_max_it in 1..1000,
 * newton_rtol in [1e-15, 1e-3] (RT_E_INVALID otherwise).  The FP64 CPU
 * reference of this library uses the defaults.  With float intensities the
 * iterate is D = T - T^n in float, every term of the energy row the size of
 * D (it is formed in deviations from each cell's smallest intensity), and
 * the tolerance is max(newton_rtol, 1e-6): the float iterate resolves D to a
 * few float ulps of D, not of T. */
typedef struct {
  int precision;
  double cfl;        /* dt = cfl * min dx / Crat when rt_step gets dt <= 0      */
  double gamma;      /* adiabatic index: E_g = rho R_ideal T / (gamma - 1)      */
  double r_ideal;
  int hold_T;        /* 1: gas temperature held fixed (secs. 5.3, 5.8)        */
  int estimate_v;    /* 1: use the sec. 4.5 half-step velocity in Steps 4-5   */
  int device_ptrs;   /* 1: array arguments are device pointers               */
  void *stream;      /* cudaStream_t the context launches on                  */
  int newton_max_it; /* iteration cap of the T^4 Newton solve                 */
  double newton_rtol;/* its stopping tolerance on |dT| / T                     */
} rt_options;

/* Fills *o with the defaults above.  RT_E_INVALID if o is NULL. */
rt_status rt_options_default(rt_options *o);

/* Writes an angle set (sec. 3) into n_out[3*m] and w_out[m] (host memory,
 * capacity `cap` angles) and its size into *m_out.  LEVEL_SYMMETRIC: the
 * LQ_N construction (Carlson 1963) with mu_1 and the class weights fixed by
 * normalisation and the even moments <mu^2k> = 1/(2k+1); the set satisfies
 * sum W = 1, sum W n = 0, sum W n n = I/3.  GAUSS_LEGENDRE: mu at the
 * Gauss-Legendre nodes, weights w_GL/2, n = (mu, sqrt(1-mu^2), 0).
 * RT_E_INVALID for an unknown kind/order or too small a capacity. */
rt_status rt_angle_set(int kind, int order, int cap, int *m_out, double *n_out, double *w_out);

/* Creates a context on the current CUDA device: validates the grid and the
 * angle set, allocates the device state (two intensity buffers of M*N
 * values, the material, T, moments and sources; about (2*M*s + 200) bytes
 * per cell, s = 8 for RT_FP64 and 4 for RT_FP32).  Crat, Prat > 0.
 * On success *out owns the state until rt_destroy. */
rt_status rt_create(const rt_grid *grid, const rt_angles *angles, double Crat, double Prat,
                    const rt_options *opts, rt_ctx **out);

/* Sets the gas fields for the following steps (sec. 2: rho, T, v; the
 * attenuation coefficients sigma_a, sigma_s).  rho, T, sigma_a, sigma_s:
 * N values; v: 3N (component-major).  Requires rho > 0, T > 0,
 * sigma >= 0, all finite (RT_E_NONFINITE / RT_E_INVALID otherwise).  The
 * first call also sets I to the isotropic equilibrium T^4/(4 pi) unless
 * rt_set_intensity was called before.  Host arrays have been read when the
 * call returns (it waits for the stream to check the values). */
rt_status rt_set_material(rt_ctx *ctx, const double *rho, const double *T, const double *v,
                          const double *sigma_a, const double *sigma_s);

/* Sets I (M*N values, angle-major).  NULL sets the isotropic equilibrium
 * I = T^4/(4 pi) from the current temperature (needs rt_set_material).
 * Recomputes E_r, F_r, P_r of the new field.  A host array has been read
 * when the call returns (it waits for the stream). */
rt_status rt_set_intensity(rt_ctx *ctx, const double *I);

/* Incoming intensities (M values) for a face with bc == RT_BC_INFLOW:
 * axis 0..dim-1, side 0 (lower) or 1 (upper).  Only rays entering the
 * domain through that face use them.  Host memory always. */
rt_status rt_set_inflow(rt_ctx *ctx, int axis, int side, const double *I_ghost);

/* Tile of cells one CTA of the step kernel owns (tx x ty x tz, one thread
 * per cell; ty = 1 for 1-D, tz = 1 below 3-D).  (0, 0, 0) restores the
 * default choice.  RT_E_INVALID when the shape is not one of the compiled
 * shapes or exceeds the 227 KB of shared memory (which grows with the angle
 * count).  Float results do not depend on the tile (bitwise); double
 * results may differ in the last bit, as the compiler fuses multiply-adds
 * differently per tile shape.  The paper has no counterpart (its code runs
 * on CPUs). */
rt_status rt_set_tile(rt_ctx *ctx, int tx, int ty, int tz);
rt_status rt_get_tile(const rt_ctx *ctx, int *tx, int *ty, int *tz);

/* Measured time of one candidate tile shape: ms per step. */
typedef struct {
  int tx, ty, tz;
  double ms;
} rt_tile_time;

/* Tile autotuner: times trial_steps (>= 1, after one untimed step) of every
 * compiled tile shape that can run this context, on its stream with CUDA
 * events, and keeps the fastest (as rt_set_tile would).  The trial steps
 * write only scratch: I, T, the moments and the step sources are restored,
 * so the state afterwards is bitwise what it was.  times (may be NULL)
 * receives up to cap entries, *ntimes (may be NULL) their count.  Waits for
 * the stream.  Needs rt_set_material and an intensity (RT_E_STATE); a
 * context in a batch is tuned through rt_batch_autotune (RT_E_STATE). */
rt_status rt_autotune(rt_ctx *ctx, int trial_steps, rt_tile_time *times, int cap, int *ntimes);

/* Step 1 of sec. 4.1: the time step cfl * min_d dx_d / Crat. */
double rt_cfl_dt(const rt_ctx *ctx);

/* One radiation step of length dt (dt <= 0: rt_cfl_dt).  Steps 2-5 of
 * sec. 4.1 plus the quadrature, fused on the device.  Updates I and T,
 * stores E_r, F_r, P_r of the new intensity and the gas sources of the step.
 * Stream-ordered: returns once the work is queued.  RT_E_STATE before
 * rt_set_material. */
rt_status rt_step(rt_ctx *ctx, double dt);

/* nsteps calls of rt_step with the same dt, launched through one captured
 * CUDA graph (no host work between steps) on a context with a stream; on
 * the legacy default stream (rt_options.stream NULL), which cannot be
 * captured, as plain launches.  The graph is kept for the next call with
 * the same dt, nsteps and buffer parity, and captured again after
 * rt_set_tile, a tile change by rt_autotune, rt_set_inflow, rt_load_state
 * or a change of the velocity terms.  RT_E_INVALID for nsteps < 0 or a non-finite dt. */
rt_status rt_run(rt_ctx *ctx, double dt, int nsteps);

/* Waits for the context's stream and reports the status of the steps run
 * since the last check: RT_E_NONFINITE if a cell's T^4 Newton iteration did
 * not converge, else RT_OK. */
rt_status rt_sync(rt_ctx *ctx);

/* E_r (N), F_r (3N), P_r (6N) of the current intensity (sec. 3 quadrature).
 * Any pointer may be NULL to skip that field.  Host pointers: the call
 * waits for the stream. */
rt_status rt_moments(rt_ctx *ctx, double *E, double *F, double *P);

/* Eddington tensor of the current intensity (sec. 2: f = K/J, the radiation
 * pressure over the energy density, f = P_r / E_r; sec. 5.2 reads f_xx and
 * f_yy of a beamed field): f[q*N + c] = P_r[q][c] / E_r[c] for q = xx, yy,
 * zz, xy, xz, yz, in double, from the stored moments; 0 where E_r = 0.
 * Host pointer (the call waits for the stream) or, with device_ptrs, a
 * device pointer.  RT_E_STATE before an intensity is set. */
rt_status rt_eddington(rt_ctx *ctx, double *f);

/* Gas sources of the last step (eqs. momentumchange, kinetichange and the
 * Delta E_T of sec. 4.3): dE_gas = Delta E_T + Delta E_K (N),
 * dMom = Delta(rho v) (3N), T_new = T^{n+1} (N).  NULL skips a field. */
rt_status rt_sources(rt_ctx *ctx, double *dE_gas, double *dMom, double *T_new);

/* One step of the loop a gas code runs around the radiation (sec. 4.1: the
 * MHD update between steps is the caller's): rt_set_material(rho, T, v,
 * sigma_a, sigma_s), rt_step(dt), rt_sources(dE_gas, dMom, T_new) in one
 * call, with the same arguments, results and errors (bitwise the same
 * outputs and state).  With host arrays the grid is cut into slabs of
 * whole tiles along its outermost active axis (z in 3-D, y in 2-D, x in
 * 1-D): the fields of a slab (and its two-plane halo) cross to the device
 * while the previous slab steps, the sources of a slab cross back while
 * the next ones step, and consecutive slabs' kernels run on two streams so
 * that one's first tiles overlap the other's last.  Other contexts (device_ptrs, bf16 storage, grids of
 * one tile layer, the first call) run the three calls in turn.
 * T_new may be T (the next step's temperature); no other output may
 * overlap an input.  Waits for the transfers.  On RT_E_NONFINITE /
 * RT_E_INVALID from the fields the intensity is unchanged and the gas
 * fields must be set again (RT_E_STATE until then). */
rt_status rt_step_coupled(rt_ctx *ctx, double dt, const double *rho, const double *T, const double *v,
                          const double *sigma_a, const double *sigma_s, double *dE_gas, double *dMom,
                          double *T_new);

/* Copies the current intensity out (M*N values, angle-major). */
rt_status rt_get_intensity(rt_ctx *ctx, double *I);

/* ---- checkpoint / resume -----------------------------------------------------
 * The restartable state of a context: the current intensity and its moments
 * in the storage type, T, the material (rho, sigma_a, sigma_s, v), the
 * inflow tables and the sources of the last step, behind a header that
 * names the grid, angle count, precision, Crat and Prat.  A fresh context
 * made by rt_create with the same grid, angles and options, loaded with
 * rt_load_state, continues bitwise as the saved one would have.  buf is
 * host memory owned by the caller.  The paper has no counterpart (its
 * restart files are Athena's). */
size_t rt_state_bytes(const rt_ctx *ctx);
/* Waits for the context's stream, then copies the state into buf (bytes >=
 * rt_state_bytes).  RT_E_STATE before rt_set_material. */
rt_status rt_save_state(rt_ctx *ctx, void *buf, size_t bytes);
/* Restores a saved state.  RT_E_INVALID when the header does not match this
 * context (grid, angle count, precision, Crat, Prat) or bytes is short;
 * RT_E_STATE for a context that belongs to a batch.  Waits for the stream. */
rt_status rt_load_state(rt_ctx *ctx, const void *buf, size_t bytes);

/* Frees the context and its device state (removing it from its batch
 * first).  NULL is ignored. */
void rt_destroy(rt_ctx *ctx);

/* ---- many problems in one launch ------------------------------------------
 * A batch advances several independent contexts together: each step is one
 * persistent kernel launch whose CTAs take (problem, tile) work items from a
 * device list, each problem with its own CFL time step.  Every problem
 * computes exactly what rt_step would give it alone.  Contexts must use
 * RT_FP32, the batch's stream, and have their material set; while in a
 * batch they are stepped only by rt_batch_step (rt_step returns
 * RT_E_STATE), and are read with the usual rt_moments / rt_sources /
 * rt_get_intensity / rt_sync calls; between steps they may take new
 * material, intensity or inflow through the usual calls.  The caller keeps
 * ownership of them. */
typedef struct rt_batch rt_batch;

/* stream: the cudaStream_t of the member contexts (NULL: legacy default
 * stream, steps launched one by one instead of through a graph). */
rt_status rt_batch_create(void *stream, rt_batch **out);
rt_status rt_batch_add(rt_batch *b, rt_ctx *ctx);
rt_status rt_batch_remove(rt_batch *b, rt_ctx *ctx);
int rt_batch_size(const rt_batch *b);
/* nsteps steps of every member, captured in one CUDA graph (one persistent
 * launch per step) when the stream is not NULL.
 * Stream-ordered.  RT_E_INVALID if the largest angle set does not fit. */
rt_status rt_batch_step(rt_batch *b, int nsteps);
/* Tile-set autotuner of the persistent kernel.  Three variants are
 * compiled: 512, 256 and 128 threads per CTA (tiles 512 / 32x16 / 16x8x4,
 * 256 / 16x16 / 8x8x4 and 128 / 16x8 / 8x4x4 cells for 1-D / 2-D / 3-D
 * members).  Times trial_steps (>= 1, after one untimed step) of each on the
 * batch's stream and keeps the fastest for later rt_batch_step calls.  The
 * members' state is restored afterwards (bitwise).  ms (may be NULL)
 * receives the three times in the order above, *chosen (may be NULL) the
 * index kept.  Waits for the stream. */
rt_status rt_batch_autotune(rt_batch *b, int trial_steps, double *ms, int *chosen);
/* Frees the batch (not its contexts).  NULL is ignored. */
void rt_batch_destroy(rt_batch *b);

/* ---- serving: continuous batching of solves ---------------------------------
 * A server runs one host thread.  rt_submit copies a request (the fields of
 * rt_create / rt_set_material, host memory, plus a step count) and returns a
 * ticket at once.  The thread admits queued requests in arrival order
 * whenever the HBM budget has room (a request that does not fit yet does not
 * block smaller ones behind it), keeps their state on the device, and
 * advances every admitted problem one step per persistent launch (rt_batch),
 * so requests arriving while others run join at the next step boundary.  A
 * finished problem's E_r, F_r, P_r are copied to host memory and its device
 * state is freed.  Requests run with RT_FP32, CFL time steps and the
 * server's options (gamma, r_ideal, hold_T, estimate_v; stream and
 * device_ptrs are the server's own).  Each result is bitwise the one the
 * problem gets alone through rt_step with the same velocity setting. */
typedef struct rt_server rt_server;
typedef long long rt_ticket;

/* hbm_budget_bytes bounds the device memory of the admitted problems (each
 * costs about 8*M + 240 bytes per cell with float intensities). */
rt_status rt_server_create(size_t hbm_budget_bytes, const rt_options *opts, rt_server **out);
/* v is 3N, the others N; nsteps >= 1.  RT_E_BUDGET if the problem alone
 * exceeds the budget, RT_E_INVALID for bad sizes or too many angles. */
rt_status rt_submit(rt_server *s, const rt_grid *grid, const rt_angles *angles, double Crat, double Prat,
                    const double *rho, const double *T, const double *v, const double *sigma_a,
                    const double *sigma_s, int nsteps, rt_ticket *out);
/* rt_submit with incoming intensities for the grid's RT_BC_INFLOW faces
 * (the sec. 5.8 beams): inflow is host memory [3][2][M] (axis, side, angle;
 * the layout of rt_noalloc_fields.inflow), read for each face whose bc is
 * RT_BC_INFLOW as rt_set_inflow would read it, or NULL (those faces then
 * let no radiation in).  RT_E_NONFINITE for a negative or non-finite
 * value.  The result is bitwise the one the problem gets alone through
 * rt_step after rt_set_inflow with the same values. */
rt_status rt_submit_inflow(rt_server *s, const rt_grid *grid, const rt_angles *angles, double Crat, double Prat,
                           const double *rho, const double *T, const double *v, const double *sigma_a,
                           const double *sigma_s, const double *inflow, int nsteps, rt_ticket *out);
/* Non-blocking.  RT_PENDING while the request is queued or running.  Once
 * it is done: RT_OK and E (N), F (3N), P (6N) copied out (NULL skips a
 * field) with the submit-to-result latency in seconds, or the request's
 * error status; either way the ticket is then released. */
rt_status rt_poll(rt_server *s, rt_ticket t, double *E, double *F, double *P, double *latency_s);
/* Blocks until the request is done (timeout_s < 0 or above 3e8 s: no
 * limit; RT_E_INVALID for NaN); RT_E_TIMEOUT when the limit passes first.
 * Does not release the ticket.  If another thread collects the ticket with
 * rt_poll during the wait, the wait returns RT_OK (the request is done).
 * No thread may wait on a server that is being destroyed. */
rt_status rt_server_wait(rt_server *s, rt_ticket t, double timeout_s);
/* Steps launched so far, requests queued / running, device bytes in use. */
rt_status rt_server_stats(rt_server *s, long long *steps, int *queued, int *running, size_t *bytes_in_use);
/* Stops the thread and frees everything, including uncollected results.
 * Servers not destroyed by the caller are destroyed when the process exits. */
void rt_server_destroy(rt_server *s);

/* ---- one step without device allocation ------------------------------------
 * The paper has no counterpart: this is a service for callers that cannot
 * allocate device memory -- code running inside another framework's memory
 * pool or under a fixed memory budget, plugins allowed to touch only the
 * buffers handed to them, and latency-critical paths where an allocation
 * could block or fail.  The caller passes every field as a device pointer;
 * the function calls no cudaMalloc, cudaFree or other allocating routine.
 * The angle and inflow tables travel in the kernel's launch parameters,
 * which limits the angle set to 256 angles (RT_E_INVALID above that).  The
 * one scratch word the step kernel needs (the count of cells whose T^4
 * Newton did not converge) is a fixed 256-byte device array that every GPU
 * loading the library holds until the process exits.
 *
 * The first call on a device looks up that array's device address (once per
 * device, with the device current); make that first call before any stream
 * capture.  Every call clears the failure word before its kernel runs, but
 * all calls share the one array: calls that overlap on the GPU (unordered
 * streams) race.
 *
 * The step is the same as rt_step with RT_FP32 and the velocity terms on
 * (grid, angles, Crat, Prat, opts->hold_T / estimate_v / gamma / r_ideal /
 * newton_max_it / newton_rtol / stream as for rt_create; opts->precision must
 * be RT_FP32; dt > 0), and gives bitwise what rt_step gives.  Layouts:
 *  - I_in, I_out: the float step's storage layout, ceil(M/4) planes of four
 *    angles each: angle m of cell c is at float index
 *    (m / 4) * 4N + 4c + (m % 4); the entries of angles M .. 4 ceil(M/4) - 1
 *    are padding (zero on input; the step writes zeros there);
 *  - rho, sigma_a, sigma_s (N floats), v (3N floats, component-major);
 *  - T (N doubles), updated in place;
 *  - mom_in, mom_out: E_r, F_r, P_r as 10N doubles in the order of
 *    rt_moments; mom_in must hold the moments of I_in;
 *  - dE_gas (N doubles), dMom (3N doubles): the step's gas sources.
 * I_in and I_out, and mom_in and mom_out, must be different buffers
 * (RT_E_INVALID when they are the same pointer): neighbouring cells read
 * the step-n values while others write the new ones.  Other overlaps
 * between the buffers are not detected and give undefined results.
 * inflow: host array [3][2][M] of incoming intensities for RT_BC_INFLOW
 * faces, or NULL.  If newton_failures is not NULL the call waits for the
 * stream and stores the number of cells whose T^4 Newton did not converge
 * (RT_E_INVALID on a stream that is being captured); otherwise it returns
 * once the work is queued. */
typedef struct {
  const float *I_in;
  float *I_out;
  const float *rho, *sigma_a, *sigma_s, *v;
  double *T;
  const double *mom_in;
  double *mom_out;
  double *dE_gas;
  double *dMom;
  const double *inflow;
} rt_noalloc_fields;

rt_status rt_step_noalloc(const rt_grid *grid, const rt_angles *angles, double Crat, double Prat,
                          const rt_options *opts, double dt, const rt_noalloc_fields *fields, int *newton_failures);

/* Message of the last failed call on this thread ("" if none). */
const char *rt_last_error(void);

/* ---- host-side fault injection (testing hook) -----------------------------
 * Makes the library's device allocation that follows `after` further
 * successful ones fail once, as if the device were out of memory: the
 * calling entry point then takes its error path (RT_E_NOMEM from rt_create,
 * an error status from rt_batch_step or a failed server request) and frees
 * what it had allocated.  kind RT_FAULT_NONE clears a pending fault.
 * RT_E_INVALID for an unknown kind or after < 0.  No GPU state is touched:
 * the failing allocation is never requested. */
enum { RT_FAULT_NONE = 0, RT_FAULT_ALLOC = 1 };
rt_status rt_fault_inject(int kind, int after);

#ifdef __cplusplus
}
#endif

#endif /* RT_GB300_H */
