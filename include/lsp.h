/*
 * lsp.h -- C ABI of the GB300 lattice Strang-splitting TDSE library.
 *
 * The library time-steps the time-dependent Schroedinger equation
 *     i gamma du/dt = -(gamma^2/2) Lap u + v u      on the d-torus [0,1)^d
 * (Suzuki, Suryanarayana, Nuyens, arXiv:1808.06357, Sec. 1 eq. TDSE) with the
 * Fourier pseudo-spectral method on a rank-1 or rank-r lattice (Sec. 2.1-2.2)
 * and Strang splitting in time (Sec. 2.3-2.5, eq. StrangTDSE, Algorithm 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: LSP_OK (0) on success, a negative LSP_ERR_* code otherwise.
 *   Nothing is thrown across the ABI.  lsp_strerror() names a code.
 * - A plan owns all device memory it uses.  Input buffers are copied; the
 *   caller keeps ownership of every pointer it passes.
 * - "on_device" arguments: 1 = the pointer is device memory on the plan's
 *   device, 0 = host memory (pageable or pinned).
 * - "stream" arguments are a cudaStream_t passed as void* (NULL = the legacy
 *   default stream).  Calls taking a stream are asynchronous on it, except
 *   that host-pointer transfers of lsp_get_state synchronise the stream
 *   before returning.  Plan creation and destruction are synchronous.
 * - One plan must not be used from two streams concurrently.
 * - State layout: u holds physical samples u(p_kappa) at the lattice points,
 *   kappa = sum_i kappa_i prod_{j>i} n_j (lexicographic, Sec. 2.5), as
 *   interleaved (re, im) pairs.  Lattice point
 *   p_kappa = (z_1 kappa_1/n_1 + ... + z_r kappa_r/n_r) mod 1 (Def. 1).
 * - Spectral layout: bin chi = sum_i xi_i prod_{j>i} n_j with
 *   xi_i = h . z_i mod n_i (Thm 1(iii), Sec. 2.5); the coefficient stored for
 *   bin chi is uhat(h_chi) = (1/n) sum_kappa u_kappa exp(-2 pi i h_chi . p_kappa)
 *   (eq. approx_uhat).
 */
#ifndef LSP_H
#define LSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsp_plan_s* lsp_plan;
typedef struct lsp_batch_s* lsp_batch;

/* Status codes. */
enum {
  LSP_OK = 0,
  LSP_ERR_BAD_ARG = -1,        /* invalid argument (null pointer, size, mode)                  */
  LSP_ERR_NOT_CANONICAL = -2,  /* lattice not in canonical form as read from Def. 1:
                                  n_{i+1} | n_i and n = prod n_i distinct points             */
  LSP_ERR_NOT_INJECTIVE = -3,  /* explicit index set violates Def. 2 or has |A| != n         */
  LSP_ERR_TOO_LARGE = -4,      /* size beyond what the kernels support                       */
  LSP_ERR_OOM = -5,            /* device allocation failed                                   */
  LSP_ERR_CUDA = -6,           /* a CUDA runtime call failed                                 */
  LSP_ERR_TIMEOUT = -7,        /* a bounded device-side wait expired; the step was abandoned */
  LSP_ERR_UNSUPPORTED = -8     /* combination not implemented (e.g. lattice shape)           */
};

/* Precision of the state and of the butterflies. */
enum { LSP_C64 = 1,  /* complex64: FP32 state, FP32 butterflies, FP64-reduced phases */
       LSP_C128 = 2  /* complex128: FP64 throughout                                  */ };

/* How the anti-aliasing set A(Z, n) of full cardinality n is chosen. */
enum { LSP_AA_MINL2 = 0,    /* each bin takes a minimal-l2 representative h_chi
                               (Lemma 4, eq. hrepresenter); computed exactly on the GPU */
       LSP_AA_EXPLICIT = 1  /* the caller supplies all n vectors h (Def. 2)             */ };

/* Space selector for lsp_get_state. */
enum { LSP_SPACE_PHYSICAL = 0, LSP_SPACE_SPECTRAL = 1 };

/*
 * lsp_plan_create -- build a plan for one TDSE instance on one device.
 *   out        receives the plan handle.
 *   d          spatial dimension, 1 <= d <= 64.
 *   r          lattice rank, 1 <= r <= 4 (r = 1: rank-1 lattice Lambda(z, n), Sec. 2.1;
 *              r >= 2: rank-r lattice Lambda(Z, n) in canonical form, Def. 1, with the
 *              r-D transform of Sec. 2.5; ranks 3 and 4 run on the SMEM-resident path).
 *   n          r moduli n_1..n_r (host); n = prod n_i points.
 *   Z          d*r generating-vector entries (host), row-major: Z[j*r + i] is
 *              component j of z_i.
 *   index_set  LSP_AA_EXPLICIT: m*d int32 entries (host), row-major, the full
 *              anti-aliasing set (m must equal n).  LSP_AA_MINL2: NULL.
 *   m          number of rows of index_set (0 for MINL2).
 *   aa_mode    LSP_AA_MINL2 or LSP_AA_EXPLICIT.
 *   prec       LSP_C64 or LSP_C128.
 *   gamma      gamma = hbar / sqrt(mass) > 0 (Sec. 1).
 *   device     CUDA device ordinal.
 * Errors: BAD_ARG, NOT_CANONICAL (n_{i+1} not dividing n_i, or fewer than n distinct
 * points), NOT_INJECTIVE, TOO_LARGE, OOM, CUDA, UNSUPPORTED; the argument, rank and
 * divisibility checks come before any device call.  On error *out is set to NULL and
 * nothing is leaked.
 * The state starts at zero and the potential at v = 0.
 * Execution paths (the first available in this order is chosen: rank 1:
 * 0, 3, 1, 4, 5, but for complex64 1, 3, 0, 4, 5 at n = 2^13, 4, 3, 0, 1, 5 from 2^20
 * to 2^24 and 3, 0, 1, 4, 5 above;
 * rank 2: 1, 2; ranks 3 and 4: 1; reported by lsp_plan_info, changed by lsp_plan_set_path or
 * lsp_plan_autotune):
 *   0 multipass, rank 1: n = 2^m, 13 <= m <= 23 (complex64) or 22 (complex128);
 *   1 SMEM-resident: any n with 2 n sizeof(complex) <= 200 KiB, any rank
 *     (rank 1 with n = 2^11 .. 2^13 (complex64) or 2^11 .. 2^12 (complex128): the
 *     state stays in registers across the steps, one line FFT per step);
 *   2 four-sweep, rank 2: (n_1, n_2) = (2^m1, 2^m2) with (m1, m2) one of
 *     (10, 8), (11, 9), (12, 10), (14, 12);
 *   3 four-sweep, rank 1: n = 2^m, m in {20, 22, 23, 24, 25};
 *   4 two-sweep with TMA-fed tiles, rank 1, complex64: n = 2^m, 16 <= m <= 24
 *     (tiles of 4096 points on 256-thread CTAs; at 2^24 of 8192 points on 512 threads);
 *   5 two-sweep with mixed-radix line transforms, rank 1: n not a power of two,
 *     n = N1 N2 with N2 <= N1 <= 4096 (eq. Fnx; any radix per factor, the four-step
 *     twiddle in FP64), chosen where no other path applies.
 * Other sizes: TOO_LARGE (rank 1) or UNSUPPORTED (ranks 2 to 4).
 */
int lsp_plan_create(lsp_plan* out, int d, int r, const int64_t* n, const int64_t* Z,
                    const int32_t* index_set, int64_t m, int aa_mode, int prec,
                    double gamma, int device);

/* Release every resource of the plan (synchronises the device). NULL is a no-op. */
void lsp_plan_destroy(lsp_plan p);

/*
 * lsp_set_potential -- v(p_kappa) for kappa = 0..n-1 as n doubles, the diagonal
 * of V_n (eq. Vn, Algorithm 1).  Copied into the plan.
 * Errors: BAD_ARG (null), CUDA.
 */
int lsp_set_potential(lsp_plan p, const double* v, int on_device, void* stream);

/*
 * lsp_set_state -- initial samples u(p_kappa), n complex values.
 *   u_prec  LSP_C64 (interleaved float pairs) or LSP_C128 (double pairs); it
 *           need not match the plan precision (converted on the device).
 * Errors: BAD_ARG, CUDA.
 */
int lsp_set_state(lsp_plan p, const void* u, int u_prec, int on_device, void* stream);

/*
 * lsp_strang_steps -- advance the state by nsteps Strang steps of size dt
 * (eq. StrangTDSE; Algorithm 1 loop body in physical space):
 *     u <- P o F^{-1} K F (P o u),  P = exp(-i dt v / (2 gamma)),
 *     K_chi = exp(-i gamma 2 pi^2 ||h_chi||^2 dt)  (eq. Fourier-ODE, eq. Dn).
 * Adjacent half potential steps are merged; the result is u at t + nsteps*dt.
 * The phase tables are rebuilt on the device from v and ||h_chi||^2 with FP64
 * argument reduction on every call.  nsteps = 0 is a no-op.
 * Errors: BAD_ARG (nsteps < 0), CUDA, TIMEOUT (returned immediately when an
 * earlier call's bounded device wait expired and no lsp_set_state followed).
 * A wait that expires during this call is reported by lsp_plan_status or the
 * next host-side lsp_get_state.
 */
int lsp_strang_steps(lsp_plan p, double dt, int64_t nsteps, void* stream);

/*
 * lsp_strang_composed -- nsteps steps of a composition of Strang steps,
 *     u <- S(w[s-1] dt) ... S(w[1] dt) S(w[0] dt) u,   S as in lsp_strang_steps,
 * for higher-order splitting (not in the paper, which names higher-order
 * splitting as future work, Sec. 5).  The symmetric triple w = (c, 1 - 2c, c),
 * c = 1 / (2 - 2^(1/3)), gives fourth order.  Each stage is a full Strang step
 * of its own size; one set of phase tables per distinct weight is built per
 * call (3 n complex of device memory for each weight after the first).
 *   nstages  1..16 stage weights in w (host).
 * Errors: BAD_ARG, OOM, CUDA, TIMEOUT (as lsp_strang_steps).
 */
int lsp_strang_composed(lsp_plan p, double dt, int64_t nsteps, int nstages, const double* w, void* stream);

/*
 * lsp_get_state -- copy the state out.
 *   out_prec  LSP_C64 or LSP_C128 element type of `out`.
 *   space     LSP_SPACE_PHYSICAL: samples u(p_kappa), kappa order;
 *             LSP_SPACE_SPECTRAL: coefficients uhat(h_chi), chi order (eq. approx_uhat).
 * Host copies synchronise `stream` before returning.
 * Errors: BAD_ARG, CUDA.
 */
int lsp_get_state(lsp_plan p, void* out, int out_prec, int space, int on_device, void* stream);

/*
 * lsp_plan_status -- synchronise `stream` and return the plan's sticky device
 * status: LSP_OK, or LSP_ERR_TIMEOUT if a bounded device-side wait of an
 * earlier lsp_strang_steps / lsp_batch_steps expired (the state is then
 * invalid until the next lsp_set_state), or LSP_ERR_CUDA.
 */
int lsp_plan_status(lsp_plan p, void* stream);

/*
 * lsp_observables -- the conserved quantities of Sec. 3.3 for the current state:
 *   out[0] = ||u_a||^2 = (1/n) sum_kappa |u_kappa|^2,
 *   out[1] = <H u_a, u_a> = sum_chi (gamma/2) 4 pi^2 ||h_chi||^2 |uhat_chi|^2
 *            + (1/gamma) (1/n) sum_kappa v_kappa |u_kappa|^2,
 * with H = -(gamma/2) Lap + v / gamma and uhat as for LSP_SPACE_SPECTRAL.  FP64
 * accumulation in a fixed order (the result does not depend on scheduling).
 * out: 2 doubles (host).  Synchronises `stream`.  Errors: BAD_ARG, OOM, CUDA, TIMEOUT.
 */
int lsp_observables(lsp_plan p, double* out, void* stream);

/* Lattice points p_kappa as n*d doubles (host), row-major (Def. 1). Errors: BAD_ARG, CUDA. */
int lsp_lattice_points(lsp_plan p, double* x);

/* ||h_chi||^2 for every bin chi, n int64 values (host) (eq. Dn / eq. hrepresenter). */
int lsp_index_norms(lsp_plan p, int64_t* norms2);

/*
 * lsp_index_table -- one representative h_chi per bin, n*d int32 values (host),
 * row-major.  MINL2 mode: a minimal-l2 vector of bin chi (eq. hrepresenter);
 * when several exist, which one is returned is unspecified but fixed.
 */
int lsp_index_table(lsp_plan p, int32_t* h);

/*
 * lsp_plan_info -- plan geometry, 8 int64 values (host):
 *   [0] n  [1] N1 (row length)  [2] N2 (column length)  [3] path (LSP_PATH_*)
 *   [4] precision  [5] device bytes held  [6] MINL2 DP box half-width (0 for
 *   EXPLICIT)  [7] max ||h_chi||^2.  For rank r >= 2, N1 = n_r (contiguous
 *   rows) and N2 = n / n_r (on the rank-2 four-sweep path, N2 = n_1).
 */
int lsp_plan_info(lsp_plan p, int64_t* info);

/* Execution paths (lsp_plan_info [3], lsp_plan_paths, lsp_plan_set_path). */
enum {
  LSP_PATH_MULTIPASS = 0,      /* rank-1, n = 2^m: two sweeps per step (persistent kernel)        */
  LSP_PATH_SMEM = 1,           /* whole run in shared memory, one CTA per instance                 */
  LSP_PATH_RANK2 = 2,          /* rank-2, 2^m1 x 2^m2: four sweeps per step                        */
  LSP_PATH_RANK1_4SWEEP = 3,   /* rank-1, n = 2^m: four sweeps per step (rows of 4096 points)      */
  LSP_PATH_RANK1_TMA = 4,      /* rank-1, n = 2^m: two sweeps per step, tiles brought in by TMA    */
  LSP_PATH_MIXED = 5           /* rank-1, n not a power of two: two sweeps, mixed-radix lines      */
};

/*
 * lsp_plan_paths -- *mask receives a bit mask of the execution paths the plan
 * can run (bit k set: path k available for its size, rank and precision).
 * Errors: BAD_ARG.
 */
int lsp_plan_paths(lsp_plan p, int* mask);

/*
 * lsp_plan_set_path -- switch the plan to an available execution path.  The
 * state, potential and ||h||^2 are kept; the path's twiddle tables are built
 * (synchronous, like plan creation).  Results of every path agree with the
 * paper's step to rounding.  A plan in a batch must keep the path it had when
 * the batch was made.  Errors: BAD_ARG, UNSUPPORTED (path not available), OOM, CUDA.
 */
int lsp_plan_set_path(lsp_plan p, int path);

/*
 * lsp_plan_autotune -- time `nsteps` Strang steps of size dt on every
 * available path and, for path 4, every kernel schedule (after one untimed call
 * of the same length), on a scratch copy of the state (the plan's state is not
 * changed), and keep the fastest path and schedule.  The decision is stored
 * (lsp_autotune_cache) and reused by later plans of the same key without
 * timing.  Not in the paper: a schedule choice.
 *   chosen  receives the kept path (may be NULL).
 *   ms      NULL, or 6 doubles (one per execution path 0..5) receiving each path's
 *           time in ms, its best schedule's for path 4 (-1: not available or not
 *           timed; path 5 is timed only for plans that no other path takes).
 * Synchronises `stream`.  Errors: BAD_ARG, OOM, CUDA, TIMEOUT (then the plan
 * keeps the path it had).
 */
int lsp_plan_autotune(lsp_plan p, double dt, int64_t nsteps, void* stream, int* chosen, double* ms);

/*
 * lsp_plan_schedule -- the plan's execution path and kernel schedule.  Path 4 has
 * three schedules, all with two CTAs per SM and potential-phase tiles brought in
 * by TMA: 0 line twiddles read where they are used; 1 each radix pass' twiddles
 * loaded before the barriers that precede the pass; 2 as 1 with the column
 * lines' twiddles in shared memory.  Other paths have one schedule (0).  Not in
 * the paper.
 *   path, sched  receive the values (either may be NULL).  Errors: BAD_ARG.
 * lsp_plan_set_schedule -- choose a schedule of the current path (results are
 * the same to rounding).  Errors: BAD_ARG, UNSUPPORTED.
 */
int lsp_plan_schedule(lsp_plan p, int* path, int* sched);
int lsp_plan_set_schedule(lsp_plan p, int sched);

/*
 * lsp_autotune_cache -- the process-wide store of autotune decisions, keyed by
 * (device name, precision, rank, moduli, available paths, step count):
 * lsp_plan_autotune on a plan whose key is stored takes the stored path and
 * schedule and its times without timing again.  clear != 0 empties the store;
 * *entries (may be NULL) receives the number of stored decisions.  Always OK.
 */
int lsp_autotune_cache(int clear, int64_t* entries);

/*
 * Batched stepping: many independent instances (same precision and device)
 * advanced together.  Instances on the SMEM-resident path run one CTA each:
 * one launch per power-of-two size on the register-resident line kernel and
 * one for all others; instances on path 4 (rank 1, 2^16 .. 2^23 points, any mix
 * of sizes, step sizes and K forms) advance together, one launch per sweep over
 * all their tiles, replayed as a CUDA graph for calls of 16 steps or more;
 * rank-1 two-sweep instances are grouped by lattice size,
 * one persistent cooperative launch per size per call; rank-1 four-sweep
 * instances of up to 2^22 points are grouped by size, one launch per sweep over
 * all the group's tiles, replayed as a CUDA graph for calls of 16 steps or more;
 * other four-sweep instances (rank 2, larger rank 1; each fills the device)
 * and path-4 instances of 2^24 points are stepped one after another.  A plan may belong to several batches, but a
 * call must not overlap another call on the same plans.
 *   lsp_batch_create  plans: `count` plan handles (host array, borrowed: the
 *                     plans must outlive the batch).  Errors: BAD_ARG, OOM, CUDA,
 *                     UNSUPPORTED (mixed precision or device).
 *   lsp_batch_steps   dt: `count` step sizes (host), one per instance;
 *                     every instance advances nsteps steps.  When an instance's
 *                     device descriptors changed since the last call (e.g. its
 *                     phase-table form), the new ones are copied on `stream`,
 *                     ordered after earlier calls on it; such a call cannot be
 *                     recorded by stream capture.  Errors as lsp_strang_steps.
 */
int lsp_batch_create(lsp_batch* out, const lsp_plan* plans, int count);
int lsp_batch_steps(lsp_batch b, const double* dt, int64_t nsteps, void* stream);
/* Synchronise `stream` and return the batch's sticky device status (as lsp_plan_status). */
int lsp_batch_status(lsp_batch b, void* stream);
void lsp_batch_destroy(lsp_batch b);

/*
 * lsp_adjoint -- gradient of a real objective J(u_T) of the final state with
 * respect to the potential samples v and the initial state u_0, by the
 * adjoint (conjugate-transposed) Strang step run backward: S^H = S(-dt),
 * since every factor of eq. StrangTDSE is unitary.  Not in the paper.
 *   dt, nsteps  as lsp_strang_steps; the plan's current state is u_0 and is
 *               left at u_T = S^nsteps u_0 on return.
 *   lamT        n complex (plan precision, device): dJ/dRe u_T + i dJ/dIm u_T.
 *   grad_v      n doubles (device): receives dJ/dv_kappa.
 *   grad_u0     n complex (plan precision, device): receives dJ/dRe u_0 + i dJ/dIm u_0.
 *   ckpt_stride steps between stored forward checkpoints (0: ceil(sqrt(nsteps))).
 * Errors: BAD_ARG, OOM, CUDA, TIMEOUT.
 */
int lsp_adjoint(lsp_plan p, double dt, int64_t nsteps, const void* lamT, double* grad_v,
                void* grad_u0, int64_t ckpt_stride, void* stream);

/*
 * lsp_strang_steps_noalloc -- nsteps Strang steps of a rank-1 lattice state,
 * like lsp_strang_steps on a plan, but allocating no device memory at all.
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc -- code under an allocator that must own every device byte, a
 * real-time or embedded loop that may not allocate once running, or a caller
 * holding no plan.  The phase and twiddle tables it needs live in one fixed
 * file-scope device array of 640 KiB that every device which loads the library
 * holds until the process exits.
 *   prec    LSP_C64 or LSP_C128 (element type of u).
 *   n       lattice size: 1 <= n <= 8192 (complex64) or <= 6400 (complex128);
 *           larger n returns LSP_ERR_TOO_LARGE.  Any factorisation of n works.
 *   gamma, dt, nsteps  as lsp_plan_create / lsp_strang_steps.
 *   v       n doubles (device): v(p_k) in point order k.
 *   norm2   n int32 (device): ||h_xi||^2 per bin xi = 0..n-1 (e.g. the values
 *           lsp_index_norms returns for the same lattice).
 *   u       n complex (device), read and overwritten in place.
 * Runs on the current CUDA device, asynchronously on `stream`.  The first call
 * on a device (nsteps = 0 is enough) looks up the device address of the array
 * (cudaGetSymbolAddress); with lazy module loading that lookup also loads the
 * library's module and so reserves the array, which can fail if the device is
 * full.  Make that first call before the allocation-free phase begins and before
 * any stream capture.  The address is kept per device for the life of the
 * process: do not call this after cudaDeviceReset on that device.  Every call
 * on a device shares the one array and rewrites it completely, so calls that
 * overlap on the GPU (other streams, other threads) race; serialise them.
 * Errors: BAD_ARG, TOO_LARGE, CUDA.
 */
int lsp_strang_steps_noalloc(int prec, int64_t n, double gamma, double dt, int64_t nsteps,
                             const double* v, const int32_t* norm2, void* u, void* stream);

/*
 * lsp_cbc_reconstructing -- a lattice on which h -> bin is injective on a given
 * index set, built component by component on the GPU (Sec. 3.1 builds the
 * paper's lattices by a component-by-component search; the acceptance test here
 * is the injectivity that Def. 2 and Thm 1(iii) ask of the anti-aliasing set).
 * Component 0 is fixed: z_0 = 1 (rank 1) or (z_{1,0}, z_{2,0}) = (1, 0) (rank 2,
 * so that (1, 0) and (0, 1) are bins and the map onto Z_n1 x Z_n2 is onto).
 * For j = 1 .. d-1 the first candidate of component j's list for which
 *   h -> (h_0..h_j).(z_0..z_j) mod n            (rank 1), or
 *   h -> ((h_0..h_j).(z_1..) mod n1) n2 + ((h_0..h_j).(z_2..) mod n2)  (rank 2)
 * is injective on the projection of I onto its first j + 1 coordinates is kept.
 * Component 0 itself is checked first (distinct values of h_0 must have distinct
 * residues mod n_1); if that fails the call returns NOT_INJECTIVE with *fixed = 0.
 * Candidates are reduced mod n_i before use and Z_out holds the reduced values.
 *   I       m x d int32 (host), row-major: the index set (rows may repeat).
 *   r       1 or 2;  n  r moduli (host), with n_1 (n_2) <= 2^31 and the bin
 *           count n (rank 1) or n_1 n_2 (rank 2) <= 2^31.
 *   cand    (d - 1) x ncand x r int64 (host): component j's candidates at
 *           cand[((j - 1) ncand + t) r .. + r), tried in order t = 0, 1, ...
 *   Z_out   d x r int64 (host), row-major: the components accepted (zeros after
 *           the first component without an injective candidate).
 *   fixed   (host, may be NULL) number of components fixed, d on success.
 *   device  CUDA device ordinal.  Synchronous; holds one 8-byte word per bin
 *           and the index set on the device while it runs.
 * Errors: BAD_ARG, NOT_INJECTIVE (no candidate of some component's list is
 * injective), OOM, CUDA, TIMEOUT (a bounded device-side retry loop gave up).
 */
int lsp_cbc_reconstructing(const int32_t* I, int64_t m, int d, int r, const int64_t* n, const int64_t* cand,
                           int64_t ncand, int64_t* Z_out, int* fixed, int device);

/*
 * lsp_sweep_times -- per-sweep durations of the multi-launch paths (2, 3, 4):
 * nsteps (2 .. 4096) Strang steps of size dt on a scratch copy of the state,
 * once untimed, then again with a CUDA event after each launch (path 4: the
 * launches and events captured into a CUDA graph and replayed, as a call of 16
 * steps or more runs; paths 2 and 3: plain launches);
 * ms[0..3] (host) = mean duration in ms of the P sweep between steps (rows /
 * X / the column sweep of path 4), the A / Y sweep, the K sweep (B / Z / the
 * row sweep of path 4) and the A^-1 / Y^-1 sweep (-1 where a path has none).
 * The plan's state is unchanged; its phase tables are rebuilt for dt.
 * Synchronous.  Errors: BAD_ARG, UNSUPPORTED (other paths), OOM, CUDA, TIMEOUT.
 */
int lsp_sweep_times(lsp_plan p, double dt, int64_t nsteps, void* stream, double* ms);

/*
 * lsp_plan_set_wait_limit -- test hook for failure detection: the number of
 * polls (~100 ns each) a bounded device-side wait of this plan's kernels (the
 * grid barrier and the tile-prefetch wait of the persistent two-sweep kernel)
 * makes before it gives up, sets LSP_ERR_TIMEOUT and returns.  0 restores the
 * default (2^25 polls, seconds).  A wait that gives up leaves no copy in flight;
 * lsp_set_state then clears the status.  Not in the paper.
 * Errors: BAD_ARG (null plan, polls < 0).
 */
int lsp_plan_set_wait_limit(lsp_plan p, int64_t polls);

/*
 * lsp_fma_rate -- measured arithmetic peak of `device` for the bound of the
 * complex128 path (prec = LSP_C128: FP64 fused multiply-adds) or of FP32 work
 * (LSP_C64): one launch of independent FMA chains on every SM, timed with CUDA
 * events after a warm-up launch.  *tflops receives flops per second / 1e12 (an
 * FMA counts 2), *ms (may be NULL) the launch time.  Synchronous; allocates one
 * word.  Not in the paper: the denominator of the complex128 roofline.
 * Errors: BAD_ARG, OOM, CUDA.
 */
int lsp_fma_rate(int device, int prec, double* tflops, double* ms);

/* Human-readable name of a status code (static storage). */
const char* lsp_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* LSP_H */
