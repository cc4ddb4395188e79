/*
 * gpsoc.h -- C ABI of the GB300 ground-state solver for rotating
 * spin-orbit-coupled spin-1 Bose-Einstein condensates (arXiv 2602.17950).
 *
 * The library minimises the discretised energy functional (Section 1, Eq. energy)
 * on the unit sphere (Eqs. groundstate, sphere) with the preconditioned nonlinear
 * conjugate gradient method (Section 3.1, Algorithms 1 and 2), the combined
 * preconditioner (Section 3.4, Eq. PreCondMix) and cascadic multigrid
 * (Section 3.3, Algorithm 3), on a periodic Fourier-spectral grid
 * (Section 3.2).  All numerical work runs in CUDA kernels on the current device.
 *
 * Conventions shared by every entry point
 *   - Wave function layout: [solve][component][z][y][x], x fastest, components
 *     ordered (phi_1, phi_0, phi_-1), each value a complex number stored as two
 *     doubles (re, im).  One solve holds 3 * nx * ny (* nz) complex values.
 *   - Grid (Section 3.2): box prod_i [-L_i, L_i], n_i even points per axis,
 *     h_i = 2 L_i / n_i, x_m = -L_i + m h_i.  The GPU FFTs need every n_i to be
 *     a power of two in [8, 1024].
 *   - Integrals are h^d times sums over grid points; <v,u> = h^d sum v conj(u).
 *   - Host pointers are owned by the caller and only read or written during the
 *     call.  Device pointers passed in are borrowed for the call only and must
 *     be valid on the problem's CUDA stream.
 *   - Every call returns a gpsoc_status; none throws.  On failure
 *     gpsoc_last_error() gives a message (thread-local, valid until the next
 *     call on that thread).
 *   - The library allocates and owns all device memory of a problem; it is
 *     released by gpsoc_destroy.
 */
#ifndef GPSOC_H
#define GPSOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GPSOC_OK = 0,
  GPSOC_EINVAL = 1,      /* invalid argument (sizes, NULL pointers, options) */
  GPSOC_ENOMEM = 2,      /* device or host allocation failed */
  GPSOC_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
  GPSOC_ENOTCONV = 4,    /* max_iter reached before the stopping criterion */
  GPSOC_ENONFINITE = 5,  /* a reduction (energy, mu, norms) became NaN or Inf */
  GPSOC_ETIMEOUT = 6,    /* a bounded host wait ran out */
  GPSOC_ESTATE = 7,      /* call made in the wrong state (e.g. solve before set_initial) */
  GPSOC_EBUDGET = 8,     /* the request does not fit the memory budget */
  GPSOC_ESTAGNATED = 9,  /* Algorithm 2 found no energy decrease (converged to rounding) */
  GPSOC_ECANCELED = 10   /* a served request was withdrawn by gpsoc_server_cancel */
} gpsoc_status;

enum { GPSOC_TRAP_HARMONIC = 0, GPSOC_TRAP_HARMONIC_QUARTIC = 1, GPSOC_TRAP_USER = 2 };
/* Precision of a solve.  FP64: every array and operation in FP64.  MIXED: an FP32
 * phase per level (FP32 arrays, FP64 sums and step decisions) until the FP32
 * rounding floor, then FP64 iterations to the stopping rule.  HYBRID: after an
 * FP64 lead-in (hybrid_lead_res), FP64 wave function, residual, reductions and
 * step decisions, with H_lin Phi advanced by linearity from an FP32 H_lin P and
 * recomputed in FP64 every hybrid_refresh iterations and before a residual is
 * accepted; the preconditioner's and the search direction's transforms run in
 * FP32.  HYBRID stops on the same FP64 rule as FP64 and reaches its fixed point. */
enum { GPSOC_FP64 = 0, GPSOC_MIXED = 1, GPSOC_HYBRID = 2 };
enum { GPSOC_STOP_DPHI = 1, GPSOC_STOP_RES = 2, GPSOC_STOP_ENERGY = 3 };
/* Preconditioner of the PCG (Section 3.4): the combined P_C = P_V^(1/2) P_Delta P_V^(1/2)
 * (Eq. PreCondMix), the kinetic P_Delta alone (Eq. PreCondKin), the potential P_V alone
 * (Eq. PreCondPot), or none (z = r). */
enum { GPSOC_PRECOND_COMBINED = 0, GPSOC_PRECOND_KINETIC = 1, GPSOC_PRECOND_POTENTIAL = 2, GPSOC_PRECOND_NONE = 3 };

/* Grid of Section 3.2.  dim = 2 or 3; n[i], L[i] for x, y(, z). */
typedef struct {
  int dim;
  int n[3];
  double L[3];
} gpsoc_grid;

/* Trapping potential V(x) (Eq. harmonic, Eq. harm-quart):
 *   V = 1/2 sum_i g[i]^2 x_i^2 + quad * r^2 + quart * r^4 (+ user_V),
 * r^2 summed over all dim axes.  HARMONIC uses g only; HARMONIC_QUARTIC adds
 * quad and quart; USER adds user_V (host array of nx*ny*nz doubles, [z][y][x],
 * copied at create; only allowed with single-level solves). */
typedef struct {
  int kind;
  double g[3];
  double quad, quart;
  const double* user_V;
} gpsoc_trap;

/* Physical parameters of one solve: rotation speed Omega, SOC strength gamma,
 * spin-independent interaction beta0 (= c0) and spin-exchange interaction
 * beta1 (= c1) (Section 1, after Eq. GPE3). */
typedef struct {
  double Omega, gamma, beta0, beta1;
} gpsoc_params;

/* Solver options.
 *   precision    GPSOC_FP64, GPSOC_MIXED or GPSOC_HYBRID (see above).
 *   stop         stopping criterion (Section 3.4, Eqs. stop1-stop3).
 *   tol          tolerance of that criterion.
 *   res_tol      if > 0, additionally require max_l ||r_l||_inf < res_tol.
 *   max_iter     iteration cap per multigrid level.
 *   theta_trial, sigma, max_halvings: Algorithm 2 (trial step, backtracking
 *                factor, cap on halvings).  Zero selects 0.1, 0.5, 40.
 *   cm_levels    1 = plain PCG on the grid; k > 1 = Algorithm 3 starting on the
 *                grid coarsened by 2^(k-1) per axis (the initial guess must then
 *                be given on that coarsest grid).
 *   check_every  iterations run between host convergence checks (0 = 16).
 *   fp32_switch  GPSOC_MIXED only: the FP32 phase of each level ends when an
 *                accepted step changes the energy by less than
 *                tol + fp32_switch * |E|, when the energy fell by less than
 *                fp32_switch * |E| per iteration on average over the last 256
 *                iterations, or when no decrease is found; 0 selects 1e-10.
 *   fp32_min_points  GPSOC_MIXED only: a level (or server bucket) whose solves x
 *                grid points fall below this runs in FP64 alone, since FP32
 *                arrays save little on work that is bound by launch latency;
 *                0 selects 65536, a negative value gives every level an FP32 phase.
 *   precond      GPSOC_PRECOND_* (0 = the combined preconditioner).
 *   fp32_res_switch  GPSOC_MIXED only: the FP32 phase of a level also ends once
 *                max_l ||r_l||_inf < fp32_res_switch, and takes no step when the
 *                level starts below it (0 = no residual rule).
 *   fp32_carry   GPSOC_MIXED only: 0 restarts the FP64 phase of a level with
 *                beta = 0; 1 continues it from the FP32 phase's last direction
 *                (beta, r_prev, P_prev carried over; measured slower on the 512^2
 *                workload, so off by default).  A solve that took no FP32 step on a
 *                level keeps its FP64 state unchanged.
 *   hybrid_refresh GPSOC_HYBRID only: iterations between exact FP64
 *                recomputations of H_lin Phi (0 = 16).
 *   hybrid_lead_res GPSOC_HYBRID only: the first (coarsest) level first runs
 *                FP64 iterations until max_l ||r_l||_inf < hybrid_lead_res (the early
 *                iterations from the initial guess decide which local minimum is
 *                reached), then the hybrid ones; finer levels are hybrid throughout.
 *                0 selects 1e-4, a negative value runs no FP64 lead-in.
 *   line_search  0: the step size of Algorithm 2 (minimiser of the quadratic model
 *                of Eqs. approeng-bn); 1: the minimiser of Eq. theta on the explicit
 *                sin/cos form of E(theta) (the first zero of dE/dtheta bracketed by
 *                doubling from the model's step, Newton steps kept in the bracket);
 *                Algorithm 2's acceptance test and halvings apply to both. */
typedef struct {
  int precision;
  int stop;
  double tol;
  double res_tol;
  int max_iter;
  double theta_trial, sigma;
  int max_halvings;
  int cm_levels;
  int check_every;
  double fp32_switch;
  int fp32_min_points;
  int precond;
  double fp32_res_switch;
  int fp32_carry;
  int hybrid_refresh;
  double hybrid_lead_res;
  int line_search;
} gpsoc_opts;

/* Per-solve result.  energy, mu, mass[] describe the final iterate;
 * res_inf = max_l ||r_l||_inf of that iterate; dE_last = energy change of the
 * last accepted step; level_iters[k] = iterations on multigrid level k
 * (k = 0 the coarsest, at most 8 levels), level_fp32_iters[k] = those of them
 * taken in FP32 arrays (GPSOC_MIXED), level_res_fp32[k] = max_l ||r_l||_inf where
 * level k's FP32 phase ended (0 if it had none). */
typedef struct {
  int status;            /* gpsoc_status of this solve */
  int iters;             /* iterations on the finest level */
  int total_iters;       /* iterations summed over levels */
  int levels;
  int beta_resets, halvings, fp32_iters, fp64_iters;
  double energy, mu, mass[3], res_inf, dE_last;
  int level_iters[8];
  int level_fp32_iters[8];
  double level_res_fp32[8];
} gpsoc_result;

typedef struct gpsoc_problem gpsoc_problem;

/* Create a problem of `batch` independent solves that share grid and trap and
 * differ in physical parameters params[0..batch-1].  cuda_stream is a
 * cudaStream_t (NULL = the library creates its own).  The grid given is the
 * finest one.  Returns EINVAL for odd or non-power-of-two sizes, L <= 0,
 * batch < 1, non-finite parameters; ENOMEM if device memory runs out. */
gpsoc_status gpsoc_create(const gpsoc_grid* grid, const gpsoc_trap* trap,
                          const gpsoc_params* params, int batch, void* cuda_stream,
                          gpsoc_problem** out);

/* Destroy a problem and free its device memory.  NULL is ignored. */
void gpsoc_destroy(gpsoc_problem* p);

/* Size in complex values of one solve's wave function on the grid of level
 * `level` (0 = finest, 1 = finest/2 per axis, ...). */
size_t gpsoc_solve_size(const gpsoc_problem* p, int level);

/* Set the initial guess of every solve from host memory (batch * 3 * npts
 * complex as interleaved doubles) on the grid of `level` (0 = finest; use
 * cm_levels - 1 for a multigrid solve).  Each solve is normalised to total
 * mass 1 (Eq. mass), keeping its component mass ratios. */
gpsoc_status gpsoc_set_initial(gpsoc_problem* p, const double* psi, int level);

/* Same from device memory (complex128, or complex64 if is_fp32). */
gpsoc_status gpsoc_set_initial_device(gpsoc_problem* p, const void* dptr, int is_fp32, int level);

/* Initial guesses (a)-(f) of Section 4: kind[c] in 0..9 = a, b, b_bar, c,
 * c_bar, d, d_bar, e, e_bar, f for component c, divided by sqrt(3) and
 * normalised; generated on the device for every solve on the grid of `level`.
 * Guess (f) requires beta0 > 0 and a harmonic trap. */
gpsoc_status gpsoc_set_initial_kind(gpsoc_problem* p, const int kind[3], int level);

/* Run Algorithm 3 (or Algorithm 1 if opts->cm_levels == 1) for every solve to
 * the stopping criterion.  results (may be NULL) receives batch entries.  The
 * call returns GPSOC_OK when every solve converged, else the first failing
 * solve's status; per-solve status is in results[]. */
gpsoc_status gpsoc_solve(gpsoc_problem* p, const gpsoc_opts* opts, gpsoc_result* results);

/* Run exactly `iters` PCG iterations on the current level and state without
 * any stopping test (restart = 1 starts with beta = 0).  For step-by-step
 * comparison with a reference implementation.  opts->precision = GPSOC_MIXED
 * runs the iterations in FP32 arrays (FP64 sums, scalars and step decisions,
 * as in the FP32 phase of a mixed solve) from the FP64 state and writes the
 * result back to it; restart = 0 continues the direction of the previous
 * gpsoc_iterate call, which must then have used the same precision. */
gpsoc_status gpsoc_iterate(gpsoc_problem* p, const gpsoc_opts* opts, int iters, int restart,
                           gpsoc_result* results);

/* Copy the current wave functions to host memory (batch * 3 * npts complex). */
gpsoc_status gpsoc_get_psi(const gpsoc_problem* p, double* psi_out);

/* Copy the current wave functions to device memory (complex128). */
gpsoc_status gpsoc_get_psi_device(const gpsoc_problem* p, void* dptr);

/* Energy (Eq. energy), chemical potential (Eq. muphi) and component masses of
 * the current iterate of every solve (arrays of length batch, mass 3*batch). */
gpsoc_status gpsoc_get_observables(gpsoc_problem* p, double* E, double* mu, double* mass);

/* Operator-level entry points (Sections 2.2, 3.1, 3.4) on the current level.
 * Host arrays as in gpsoc_set_initial.  precision = GPSOC_FP64 runs the FP64
 * kernels; GPSOC_MIXED runs the FP32 kernels of the mixed-precision phase on an
 * FP32 copy of the state (FP32 transforms and pointwise work, FP64 block and
 * grid sums and scalars) and widens the array results to FP64.
 *   gpsoc_apply_h: H_l(Phi) of Eqs. eigen1-eigen3 for the current state into
 *     hpsi (may be NULL); obs (may be NULL) receives per solve 9 doubles:
 *     E, mu, alpha_1, alpha_0, alpha_-1 (Eq. PreCnstAlpha), mass_1, mass_0,
 *     mass_-1, <H_lin Phi, Phi>.
 *   gpsoc_apply_precond: P_C r (Eq. PreCondMix) for the current state's alpha
 *     and density, r given per solve; result into out.
 *   gpsoc_step_model: for directions P (one per solve, tangent or not), the
 *     coefficients a_n, b_n (Eqs. an, bn; H_l(P) read with the density frozen at
 *     Phi) and the energy change E(cos t Phi + sin t P/||P||) - E(Phi) at
 *     n_theta angles theta[]; out receives per solve 2 + n_theta doubles. */
gpsoc_status gpsoc_apply_h(gpsoc_problem* p, int precision, double* hpsi, double* obs);
gpsoc_status gpsoc_apply_precond(gpsoc_problem* p, int precision, const double* r, double* out);
gpsoc_status gpsoc_step_model(gpsoc_problem* p, int precision, const double* P, const double* theta, int n_theta,
                              double* out);

/* Spectral zero-padding prolongation (Section 3.3, step c; read as zero
 * padding) of every solve from level `level` to level `level - 1`, followed by
 * renormalisation to unit mass; the result becomes the current state. */
gpsoc_status gpsoc_prolong(gpsoc_problem* p, int level);

/* Batched 1-D FFTs along one axis (axis 0 = x, 1 = y, 2 = z) of `count`
 * arrays laid out like one component on the problem's finest grid, in place on
 * device memory `data` (complex128).  inverse != 0 applies the inverse
 * transform including 1/n (Section 3.2 convention, forward unnormalised). */
gpsoc_status gpsoc_fft_axis(gpsoc_problem* p, void* data, int count, int axis, int inverse);

/* Served form: continuous batching of ground-state requests (the paper's method
 * applied to a stream of independent problems; no counterpart in the paper).
 * Requests are grouped by grid, trap and stopping rule into buckets of
 * slots_per_bucket solves that advance together in rounds of iters_per_step PCG
 * iterations (one CUDA graph replay per two iterations), each bucket on its own
 * stream and at its own pace.  gpsoc_server_step retires the solves that stopped
 * in every bucket whose round has finished (waiting for the earliest-launched
 * round if none has), refills free slots from the queue in arrival order, and
 * starts the next round of every idle bucket that holds work; it returns while
 * rounds run.  Buckets are created while hbm_budget_bytes allows and released
 * when empty, idle and the room is needed.  With GPSOC_MIXED a request runs first in FP32 arrays (FP64
 * sums) and then in FP64 from that iterate to its stopping rule.  Requests are
 * single-level solves (opts->cm_levels must be 0 or 1) with analytic traps. */
typedef struct gpsoc_server gpsoc_server;
typedef struct {
  double hbm_budget_bytes;   /* device memory the buckets may use */
  int slots_per_bucket;      /* solves per bucket (0 = 32) */
  int precision;             /* GPSOC_FP64 or GPSOC_MIXED */
  int iters_per_step;        /* PCG iterations per bucket and step (0 = 32) */
} gpsoc_server_opts;

gpsoc_status gpsoc_server_create(const gpsoc_server_opts* opts, gpsoc_server** out);
void gpsoc_server_destroy(gpsoc_server* s);
/* Queue one request: psi0 is the host initial guess on the grid (3 * npts complex,
 * normalised on admission); the arguments are copied.  *ticket identifies it. */
gpsoc_status gpsoc_server_submit(gpsoc_server* s, const gpsoc_grid* grid, const gpsoc_trap* trap,
                                 const gpsoc_params* params, const double* psi0, const gpsoc_opts* opts,
                                 uint64_t* ticket);
/* Retire, admit, launch (see above).  *busy (may be NULL) receives the number of
 * requests queued or running.  Not thread-safe: one caller per server. */
gpsoc_status gpsoc_server_step(gpsoc_server* s, int* busy);
/* Result of one request.  timeout_ms = 0 only looks; timeout_ms > 0 drives the
 * server (gpsoc_server_step) until the request finishes or timeout_ms have
 * passed, waiting on the device in steps of at most that bound; timeout_ms < 0
 * drives it until the request finishes.  Returns GPSOC_OK with the result (and
 * the final wave function in psi_out, may be NULL) once the request finished --
 * the ticket is then released; GPSOC_ETIMEOUT while it is still queued or
 * running; GPSOC_EINVAL for an unknown ticket.  A cancelled request reports
 * GPSOC_OK with res->status = GPSOC_ECANCELED and leaves psi_out untouched. */
gpsoc_status gpsoc_server_poll(gpsoc_server* s, uint64_t ticket, int timeout_ms, gpsoc_result* res,
                               double* psi_out);
/* Withdraw a queued or running request.  A running solve is stopped on the device
 * after the round in flight (stream-ordered) and its slot is freed at once; the
 * ticket then polls as finished with status GPSOC_ECANCELED.  GPSOC_ESTATE if the
 * request has already finished, GPSOC_EINVAL for an unknown ticket. */
gpsoc_status gpsoc_server_cancel(gpsoc_server* s, uint64_t ticket);
/* Device bytes reserved by buckets, number of buckets, queued requests. */
gpsoc_status gpsoc_server_stats(const gpsoc_server* s, double* bytes_in_use, int* buckets, int* queued);

/* Instrumentation (no counterpart in the paper; used by the benchmark).
 *   gpsoc_profile: run `iters` PCG iterations from the current state (beta
 *     restarted, no stopping test) with a CUDA event recorded after every
 *     kernel on the problem's stream; ms[k] receives the average duration of the
 *     k-th kernel of an iteration (at most cap entries), *n_kernels the number
 *     of kernels per iteration.  The state advances by `iters` iterations.
 *   gpsoc_profile_name: name of the k-th kernel of the last profile ("" if none).
 *   gpsoc_kernel_launches: number of kernels this problem has launched so far
 *     (each replay of a captured iteration graph counts all its kernels). */
gpsoc_status gpsoc_profile(gpsoc_problem* p, const gpsoc_opts* opts, int iters, double* ms, int cap, int* n_kernels);
const char* gpsoc_profile_name(const gpsoc_problem* p, int k);
uint64_t gpsoc_kernel_launches(const gpsoc_problem* p);
/* Tile of the FFT passes along `axis` (0 = x rows, 1 = y, 2 = z columns) on
 * multigrid level `level` for this problem's batch in the given precision:
 * *lines = grid lines per thread block (rows for x, adjacent columns for y, z),
 * *elems_per_thread = FFT elements per thread (the radix of the Stockham
 * passes), *threads = threads per block. */
gpsoc_status gpsoc_tile_shape(const gpsoc_problem* p, int level, int axis, int precision, int* lines,
                              int* elems_per_thread, int* threads);

/* Tile autotuning (no counterpart in the paper).  Tiles are chosen per grid,
 * batch size and kernel precision (FP64 kernels for GPSOC_FP64, FP32 kernels for
 * GPSOC_MIXED and GPSOC_HYBRID) from a process-wide table; keys without an entry
 * use the built-in rule (the largest tile that still gives at least two blocks
 * per SM).  Every problem with the same grid, batch and precision uses the table
 * entry, which sets all passes along an axis together.
 *   gpsoc_tile_candidates: the valid (lines, elems_per_thread) tiles of an axis on
 *     a level: lines a power of two, elems_per_thread a supported radix (2, 4, 8,
 *     and 16 for FP32 column passes), at most 384 threads and 200 KB of shared
 *     memory per block.  Writes min(count, cap) pairs; *count = all of them.
 *   gpsoc_tuning_set: set the tile of an axis for this problem's grid (at `level`),
 *     batch and precision; lines = 0 returns the axis to the rule; EINVAL if the
 *     tile is not a candidate.  The problem's captured graphs are dropped.
 *   gpsoc_autotune: on the current level, time every candidate of each axis
 *     (CUDA events over `iters` profiled iterations of opts->precision, each from
 *     the same state) against the rule and keep the fastest; lines[3] and
 *     elems_per_thread[3] (may be NULL) receive the tiles now in use (0 beyond
 *     dim).  The state is restored afterwards but iteration counters are reset. */
gpsoc_status gpsoc_tile_candidates(const gpsoc_problem* p, int level, int axis, int precision, int* lines,
                                   int* elems_per_thread, int cap, int* count);
gpsoc_status gpsoc_tuning_set(const gpsoc_problem* p, int level, int axis, int precision, int lines,
                              int elems_per_thread);
gpsoc_status gpsoc_autotune(gpsoc_problem* p, const gpsoc_opts* opts, int iters, int* lines, int* elems_per_thread);

/* Arithmetic roofline probe (no counterpart in the paper): FP64 and FP32 FMA
 * throughput of the current device in TFLOP/s (an FMA counts 2 flops), from
 * independent FMA chains run for a few milliseconds.  Either pointer may be NULL. */
gpsoc_status gpsoc_probe_peaks(double* fp64_tflops, double* fp32_tflops);

/* Allocation-free H(Phi) (no counterpart in the paper).  For callers that must
 * not allocate device memory when they need the Hamiltonian -- a framework that
 * owns all device memory through its own pool, a real-time loop that cannot
 * afford (or synchronise on) cudaMalloc/cudaFree, code held to a memory budget
 * reserved up front.  Computes what gpsoc_apply_h computes, H_l(Phi) of
 * Eqs. eigen1-eigen3 and the 9 observables per solve, without a problem object:
 *   grid, trap (HARMONIC or HARMONIC_QUARTIC), params[batch]: as gpsoc_create;
 *   d_psi:  device, batch * 3 * npts complex128, [solve][component][z][y][x],
 *           used as given (not normalised), read only;
 *   d_hpsi: device, same layout, receives H_l(Phi);
 *   obs:    host, 9 doubles per solve as gpsoc_apply_h (may be NULL);
 *   cuda_stream: cudaStream_t or NULL (legacy default stream); the call
 *           returns after the stream has finished its work.
 * It allocates nothing: intermediate arrays, partial sums, twiddle tables and
 * per-solve scalars live in one fixed 16 MiB array in device memory, present on
 * every GPU that loads the library until the process exits.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) and sets
 * kernel attributes; make that first call before any stream capture.  Problems
 * whose working set (about 4 x batch x 3 x npts x 16 bytes plus small tables)
 * exceeds the array return GPSOC_EBUDGET.  Failures are reported by the
 * returned status only (gpsoc_last_error is not updated: that would allocate a
 * message).  All calls share the one array: calls
 * whose work overlaps on the GPU (other threads, other streams) race and must
 * be serialised by the caller. */
gpsoc_status gpsoc_apply_h_noalloc(const gpsoc_grid* grid, const gpsoc_trap* trap, const gpsoc_params* params,
                                   int batch, const void* d_psi, void* d_hpsi, double* obs, void* cuda_stream);

/* Message describing the last failure on this thread ("" if none). */
const char* gpsoc_last_error(void);

/* Library version string. */
const char* gpsoc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GPSOC_H */
