/*
 * dyson.h -- C ABI of the GB300 solver for the diagonal of the lattice
 * Green's function of inhomogeneous DMFT,
 *
 *     G_ii(i w_k) = [H(i w_k)^-1]_ii,
 *     H_ij(i w_k) = t_ij + (i w_k + mu - V_i - Sigma_i(i w_k)) delta_ij,
 *
 * (Eq. 1 of Carrier, Tang, Saad, Freericks, "Lanczos-based Low-Rank Correction
 * Method for Solving the Dyson Equation in Inhomogeneous Dynamical Mean-Field
 * Theory", and the text after it: t_ij = t on nearest neighbours of a square
 * or simple-cubic lattice, H complex symmetric with real off-diagonals; only
 * diag(G) is wanted, Sec. 1 end).  The diagonal is computed by the paper's
 * Lanczos-based low-rank correction method (Sec. 2.3, Eqs. 5-9):
 *
 *     diag(H^-1) = diag(blkdiag(B^-1, 0)) + diag(Q_k T_k Q_k^T),
 *
 * B the subdomain blocks of the domain-decomposition ordering (Sec. 2.2,
 * Eq. 3) and Q_k T_k Q_k^T the rank-k complex-symmetric Lanczos
 * approximation of X = H^-1 - blkdiag(B^-1, 0) (Eq. 6, Eq. 10).
 *
 * Conventions shared by every call
 *   - Sites are in natural order, x fastest: i = x + Lx*(y + Ly*z).
 *   - Complex numbers are interleaved (re, im) pairs of double (layout of
 *     C99 double _Complex); "complex[K][N]" is K*N such pairs, row-major.
 *   - Boundaries are open on every axis.
 *   - Domain decomposition: the slowest axis (y in 2D, z in 3D) is cut into
 *     p strips/slabs separated by p-1 single interface lines/planes; the first
 *     (L_slow - p + 1) mod p strips are one layer taller.  m = (p-1)*(sites
 *     per layer) interface sites.  p = 1 means no interface: the result is the
 *     exact diagonal.
 *   - mem_kind says where the caller's buffers live: DYSON_MEM_HOST (plain or
 *     pinned host memory; the call copies in, computes, copies out and returns
 *     after the stream has finished) or DYSON_MEM_DEVICE (device pointers on
 *     the plan's device; the call only enqueues work on `stream` and returns).
 *   - stream is a cudaStream_t (NULL = the legacy default stream).
 *   - Ownership: the caller owns every buffer it passes and keeps it valid
 *     until the work on `stream` has finished; the library borrows inputs
 *     for the duration of the call and never frees them.  A plan owns its
 *     device workspace (factors, Lanczos vectors, scratch).
 *   - Errors: every call returns DYSON_OK (0) or a negative DYSON_E_* code and
 *     sets a thread-local message readable with dyson_last_error().  The
 *     library never aborts the process and its kernels never trap.
 */
#ifndef DYSON_H
#define DYSON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define DYSON_OK 0
#define DYSON_E_BAD_ARG (-1)      /* an argument is out of range or NULL */
#define DYSON_E_OOM (-2)          /* device allocation failed */
#define DYSON_E_CUDA (-3)         /* a CUDA runtime call failed */
#define DYSON_E_UNSUPPORTED (-4)  /* valid input this build does not handle */
#define DYSON_E_BUDGET (-5)       /* serving: request larger than the memory budget */
#define DYSON_E_NOT_FOUND (-6)    /* serving: unknown ticket */

/* per-frequency status flags, written to status[K] by dyson_solve */
#define DYSON_ST_OK 0
#define DYSON_ST_TERMINATED 1     /* Lanczos reached an invariant subspace before k_max: exact */
#define DYSON_ST_BREAKDOWN 2      /* (r, r)_C vanished for r != 0 (Sec. 2.1); partial sum kept */
#define DYSON_ST_NO_CONVERGENCE 4 /* an interface solve hit krylov_maxit */
#define DYSON_ST_WAIT_TIMEOUT 16  /* a bounded device wait (copy ring) gave up after 2 s: the
                                     kernel went on without hanging, the frequency's result is
                                     not valid */

/* precision forms */
#define DYSON_FP64 0   /* every step in complex128 */
#define DYSON_MIXED 1  /* sweeps, inner interface solves and the preconditioner in complex64
                          with FP32 accumulation, every solve refined against FP64 residuals;
                          diag(B^-1) from a double-float (two binary32, ~47-bit) recursion;
                          the Lanczos step's re-orthogonalisation in double-float arithmetic
                          on a double-float basis (k_max <= 64, scalar Lanczos; binary64
                          otherwise), its scalars, T_k and the diagonal in binary64.  Within
                          ~1e-6 of DYSON_FP64 where the truncated result is not amplified by
                          rounding */

/* interface preconditioner of the H solves (dyson_geometry.precond) */
#define DYSON_PRECOND_AUTO 0    /* exact layer blocks where they apply, else banded */
#define DYSON_PRECOND_BANDED 1  /* banded approximation of each layer block of S */
#define DYSON_PRECOND_LAYER 2   /* exact layer blocks S_ll (2D strips, Lx <= 160, slice width <= 32) */

#define DYSON_MEM_HOST 0
#define DYSON_MEM_DEVICE 1

typedef struct dyson_plan_s* dyson_plan;

/* Lattice, physics constants and method sizes of one plan. */
typedef struct {
  int dim;            /* 2 (square lattice) or 3 (simple cubic) */
  int L[3];           /* Lx, Ly, Lz; Lz ignored when dim == 2 */
  double t;           /* nearest-neighbour hopping t_ij */
  double mu;          /* chemical potential */
  int p;              /* subdomains along the slowest axis, 1..16 */
  int k_max;          /* Lanczos rank cap k, 1..256 (Sec. 2.3 stopping rule) */
  int precision;      /* DYSON_FP64 or DYSON_MIXED */
  double krylov_tol;  /* relative residual of each interface solve; 0 = default
                         (1e-13 FP64, 1e-5 mixed inner solves) */
  int krylov_maxit;   /* iteration cap of each interface solve; 0 = default (1000) */
  double refine_tol;  /* mixed form: relative FP64 residual after refinement; 0 = 1e-13,
                         the FP64 form's own interface tolerance (refinement also stops
                         once a pass no longer shrinks the residual 4-fold: the FP64
                         rounding floor) */
  int refine_max;     /* mixed form: most refinement passes per solve; 0 = default (6) */
  int max_freqs;      /* most frequencies one dyson_solve call may carry (>= 1) */
  double eta;         /* frequency axis.  0: Matsubara, H_ii = i w_k + mu - V_i - Sigma_i
                         (Eq. 1).  > 0: real axis, i w_k -> w + i eta (the retarded form
                         Sec. 2 notes after Eq. 1); omega[] then holds real frequencies w
                         and Sigma the retarded self-energy (Im Sigma <= 0 keeps Im H_ii >=
                         eta > 0, which the factorization relies on).  Must be >= 0. */
  int block_size;     /* Lanczos block size nb.  0 or 1: the scalar recurrence of Sec. 2.1.
                         2..4: block Lanczos on X (not in the paper): nb start vectors, A_j =
                         Q_j^T X Q_j and B_j in the bilinear form, deflation of vanishing
                         columns; reaches the exact diagonal when X has eigenvalues of
                         multiplicity up to nb, which the scalar method cannot.  k_max counts
                         columns (k_max / nb block steps) and must be a multiple of nb with
                         k_max * nb <= 1024; max_freqs * nb <= 65535. */
  int precond;        /* DYSON_PRECOND_*: preconditioner of the interface system S y = r (Eq. 4;
                         the paper leaves the solver open).  LAYER inverts the exact diagonal
                         blocks S_ll = C_ll - t^2 (surface Green's functions of the two strips
                         along line l), computed in complex64 once per solve; only the coupling
                         between different lines is left out, so COCG needs one or two
                         iterations.  BANDED keeps the entries of S_ll within two sites.
                         LAYER where it does not apply: DYSON_E_UNSUPPORTED. */
  int freq_groups;    /* frequencies of a solve are split into this many contiguous groups
                         (0: default, one group per 16 frequencies of max_freqs in the mixed
                         form and per 8 in FP64, between 1 and 4; at most 8; 1: one batch),
                         each run as its own branch
                         of the solve's CUDA graph on its own stream, the lowest-index group
                         at the highest stream priority.  Frequencies stay independent, so
                         results do not depend on the grouping.  Plans whose slice width
                         exceeds 64 always use one batch; the serving loop takes 0 as 1. */
} dyson_geometry;

/* Library version string. */
const char* dyson_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* dyson_last_error(void);

/*
 * Domain-decomposition ordering (Sec. 2.2, Fig. 1 right; Eq. 3), host only,
 * no GPU needed.  heights[p] receives the strip/slab heights along the slow
 * axis; *m the number of interface sites; if dd2nat is not NULL it receives
 * the natural site index of every slot of the internal subdomain-first
 * vector layout (length *ndd, -1 on padding slots; call once with
 * dd2nat = NULL to learn *ndd).
 */
int dyson_partition(const dyson_geometry* geom, int* heights, int* m, int* ndd, int* dd2nat);

/* Device bytes a plan for `geom` allocates (for admission by memory footprint). */
int dyson_plan_footprint(const dyson_geometry* geom, size_t* bytes);

/*
 * Create a plan on the current CUDA device: validates geom, builds the
 * domain-decomposition maps and allocates all device workspace for up to
 * geom->max_freqs frequencies.  *out is set on success.
 * Slice width W = (sites of one slice: h in 2D, Ly*h in 3D, h the tallest
 * subdomain) rounded up to a multiple of 4 must be <= 320, and, with p > 1,
 * for W > 64 the sweep row buffer (Lx * W complex entries in the form's
 * precision) must leave room for the copy ring in shared memory; otherwise
 * DYSON_E_UNSUPPORTED.  With p = 1 the solve is the exact slice recursion
 * (no interface, no sweeps), so only the width limit applies; the sweep
 * entry points (dyson_subdomain_solve, dyson_xmatvec) then check it per call.
 */
int dyson_plan_create(const dyson_geometry* geom, dyson_plan* out);

/* Free a plan and its device memory (waits for its pending work). */
int dyson_plan_destroy(dyson_plan plan);

/*
 * Autotuner result (batched kernels' tile choice).  At a plan's first
 * dyson_solve with p > 1, before its graph is captured, the library times one
 * X-matvec launch for each configuration the geometry admits -- copy-ring
 * slots, rows per streamed chunk when W > 64, and for the mixed form's
 * complex64 two-chain sweeps (W <= 64) the CTA size, 256 threads at two CTAs
 * per SM or 128 threads at four -- on the caller's inputs and keeps the
 * fastest.  Reports the configuration in use (*ring_slots, *chunk_rows,
 * *threads), how many were timed (*candidates, 0 before the first solve) and
 * the launch times of the heuristic's choice and of the kept one (ms).  Any
 * output pointer may be NULL.  The paper has no counterpart.
 */
int dyson_plan_tuning(dyson_plan plan, int* ring_slots, int* chunk_rows, int* candidates,
                      float* ms_heuristic, float* ms_best, int* threads);

/*
 * diag(G(i w_k)) for K frequencies (Eq. 1 solved by the method of Sec. 2.3):
 *   omega  [K]         real Matsubara frequencies w_k
 *   V      [N]         real local potential V_i
 *   sigma  complex[K][N]  self-energy Sigma_i(i w_k)
 *   q1     [nb][N]     real Lanczos start vector(s), nb = block_size (normalised
 *                      internally in the bilinear form; the nb columns of a
 *                      block must be independent in it, else the frequency
 *                      reports DYSON_ST_BREAKDOWN); the paper leaves it open
 *   diagG  complex[K][N]  output G_ii(i w_k)
 *   status [K]         output DYSON_ST_* flags per frequency (may be NULL)
 * All frequencies run in one batch: one thread-block cluster per frequency
 * with one CTA per subdomain, the whole sequence replayed from a CUDA graph.
 * Frequencies are independent: a frequency's result does not depend on which
 * other frequencies share the call.
 */
int dyson_solve(dyson_plan plan, int K, const double* omega, const double* V,
                const double* sigma, const double* q1, double* diagG, int* status,
                int mem_kind, void* stream);

/*
 * Diagnostics of the last dyson_solve on this plan (host buffers, each may be
 * NULL; waits for the plan's work): alpha_beta complex[K][k_max][2] holds
 * (alpha_j, beta_j) with beta_j coupling q_{j-1} and q_j (beta_1 = 0);
 * steps[K] the Lanczos steps taken; iters[K] the interface Krylov iterations
 * summed over all solves; refines[K] the refinement passes (mixed form).
 */
int dyson_solve_info(dyson_plan plan, int K, double* alpha_beta, int* steps, int* iters,
                     int* refines);

/*
 * Block plans (block_size nb >= 2): the block tridiagonal T of the last
 * dyson_solve.  AB complex[K][k_max/nb][2][nb][nb] (host) receives per block
 * step j the diagonal block A_j (row-major, A_j[d][c] = q_{j,d}^T X q_{j,c})
 * and the coupling B_j (upper triangular, R_{j-1} = Q_j B_j; B_0 = 0);
 * steps[K] the block steps taken.  dyson_solve_info's alpha_beta must be NULL
 * for block plans (its steps count block steps).  Either pointer may be NULL.
 */
int dyson_block_info(dyson_plan plan, int K, double* AB, int* steps);

/*
 * y = H(i w_k) x for K frequencies by the nearest-neighbour stencil (Eq. 1),
 * H never stored.  x, y complex[K][N] (complex128).  With DYSON_MEM_DEVICE all
 * inputs are read in place and K may exceed the plan's max_freqs; with host
 * buffers they are staged through the plan (K <= max_freqs).
 */
int dyson_apply_H(dyson_plan plan, int K, const double* omega, const double* V,
                  const double* sigma, const double* x, double* y, int mem_kind, void* stream);

/* The same product in complex64: x, y are interleaved float pairs [K][N]. */
int dyson_apply_H_c64(dyson_plan plan, int K, const double* omega, const double* V,
                      const double* sigma, const float* x, float* y, int mem_kind,
                      void* stream);

/*
 * diag(blkdiag(B^-1, 0)) per frequency (the first term of Eq. 9; Sec. 2.3:
 * computed once before the Lanczos steps) by the block-tridiagonal recursion
 * of each subdomain.  diagB complex[K][N], zero on interface sites.  Runs in
 * the plan's precision.
 */
int dyson_subdomain_diag(dyson_plan plan, int K, const double* omega, const double* V,
                         const double* sigma, double* diagB, int mem_kind, void* stream);

/* w = blkdiag(B^-1, 0) q (Eq. 7) for complex[K][N] q and w. */
int dyson_subdomain_solve(dyson_plan plan, int K, const double* omega, const double* V,
                          const double* sigma, const double* q, double* w, int mem_kind,
                          void* stream);

/*
 * u = X q = H^-1 q - blkdiag(B^-1, 0) q, the modified Lanczos "matvec" of
 * Eqs. 6-8, for complex[K][N] q and u.  FP64 form: u from the elimination
 * y = S^-1 (E^T B^-1 q_B - q_C), u_B = B^-1 E y, u_C = -y, with S applied
 * implicitly (never formed).  Mixed form: v = H^-1 q and w refined in FP64,
 * u = v - w.
 */
int dyson_xmatvec(dyson_plan plan, int K, const double* omega, const double* V,
                  const double* sigma, const double* q, double* u, int mem_kind, void* stream);

/*
 * Recursive decomposition (Sec. 2.3, last paragraph), square lattices (dim 2):
 * the lattice is cut in two by one interface line, each half across the other
 * axis, and so on, the number of domains alternating (d_x, d_y) = (2, 1),
 * (1, 2), (2, 1), ... level by level (first_cut DYSON_CUT_X; DYSON_CUT_Y
 * starts with (1, 2)).  A box (the principal submatrix H_box of H on its
 * sites, open at its edges) gets
 *     [diag of each half's inverse, by the same rule one level down; 0 on the
 *      cut line] + diag(Q_k T_k Q_k^T),
 * the rank-k Lanczos approximation (Eq. 10) of X_box = H_box^-1 -
 * blkdiag(H_1^-1, H_2^-1, 0) (Eqs. 5-8 on the box) started from q1 restricted
 * to the box.  The line sits at the middle site of the cut axis; with an even
 * extent the half before it is one site shorter.  An axis shorter than 3
 * sites is not cut (the other one is); boxes of at most min_sites sites, or
 * shorter than 3 along both axes, are inverted exactly.  The paper states
 * only the alternation; these rules are this library's reading.
 *
 * dyson_recursive_plan_create: from geom it reads L (dim must be 2), t, mu,
 * k_max (the rank cap of every box), precision, eta, krylov_tol/maxit,
 * refine_tol/max, precond, freq_groups and max_freqs; p and block_size are
 * not used (block_size must be 0 or 1).  It builds the box tree and one
 * ordinary plan per box shape and stream (streams: boxes of one level run
 * concurrently on up to this many streams, 0 = 4, at most 16), all device
 * memory allocated here.  Every box must fit an ordinary plan: its slow-axis
 * extent (the cut axis) at most 641, its leaves' shorter extent at most 320.
 * Errors: DYSON_E_BAD_ARG (dim != 2, min_sites < 1, first_cut, block_size,
 * streams, k_max or max_freqs out of range), DYSON_E_UNSUPPORTED or
 * DYSON_E_OOM from a box plan (the message names the box shape).
 *
 * dyson_recursive_solve: diag(G) for K <= max_freqs frequencies, arguments as
 * dyson_solve (q1 [N] real).  status[K]: DYSON_ST_NO_CONVERGENCE, _BREAKDOWN
 * and _WAIT_TIMEOUT of any box OR-ed; DYSON_ST_TERMINATED only when every box
 * terminated, in which case the result is the exact diagonal.  With
 * DYSON_MEM_DEVICE every buffer must be device (or managed) memory of the plan's
 * device (checked before any work: DYSON_E_BAD_ARG) and the call only enqueues
 * on `stream`; the plan's own streams wait for it and it waits for them.  Calls on one recursive plan must not
 * overlap on the GPU (they share the box plans).
 *
 * dyson_recursive_plan_info: levels of the tree, internal boxes, leaves,
 * ordinary plans created and device bytes held (each pointer may be NULL).
 *
 * dyson_recursive_boxes: the box tree alone, host only (no GPU needed).  *n
 * receives the number of boxes; if boxes is not NULL it receives, per box,
 * level by level, 8 ints: x0, y0, nx, ny (origin and extents), level, leaf
 * (1: inverted exactly), the cut axis (0: the line is the column x = line,
 * 1: the row y = line; -1 for a leaf) and the line's coordinate (-1 for a
 * leaf).  Call once with boxes = NULL to learn *n.
 */
#define DYSON_CUT_X 0
#define DYSON_CUT_Y 1
typedef struct dyson_rplan_s* dyson_rplan;
int dyson_recursive_plan_create(const dyson_geometry* geom, int min_sites, int first_cut, int streams,
                                dyson_rplan* out);
int dyson_recursive_plan_destroy(dyson_rplan rplan);
int dyson_recursive_boxes(const dyson_geometry* geom, int min_sites, int first_cut, int* n, int* boxes);
int dyson_recursive_plan_info(dyson_rplan rplan, int* levels, int* boxes, int* leaves, int* plans,
                              size_t* bytes);
int dyson_recursive_solve(dyson_rplan rplan, int K, const double* omega, const double* V,
                          const double* sigma, const double* q1, double* diagG, int* status,
                          int mem_kind, void* stream);

/*
 * Serving: continuous batching of Dyson solves from many IDMFT clients (each
 * self-consistency iteration needs all frequencies again with a new
 * self-energy, Sec. 3).  Requests are admitted in arrival order as soon as the
 * device-memory budget (bytes of resident plans) and a stream slot allow;
 * while the oldest request waits for memory, later requests whose plan is
 * resident and idle run in its place (at most 64 per waiting request).
 * Queued requests with the geometry of an admitted one and bitwise the same V
 * and start vector(s) join its solve as further frequencies, while they fit
 * the plan's max_freqs (at most 32 requests per solve): requests of uneven K
 * share one batched launch sequence.
 * Admitted requests run concurrently, each as one batched, graph-replayed
 * solve on its own stream.  Plans (factors, Lanczos bases, workspace) stay
 * resident and are reused by later requests with the same geometry; idle
 * plans are evicted least recently used first when memory is needed and
 * evicting them makes enough room.  A
 * request's result is the same alone and in any mix.  Thread-safe: any
 * thread may submit, poll and wait.
 */
typedef struct dyson_server_s* dyson_server;

typedef struct {
  dyson_geometry geom;   /* geometry and sizes; geom.max_freqs is the plan's capacity */
  int K;                 /* frequencies in this request (>= 1); more than geom.max_freqs run as
                            consecutive chunks of max_freqs on the same plan and stream */
  const double* omega;   /* [K] host (pinned host memory lets the copies overlap) */
  const double* V;       /* [N] host */
  const double* sigma;   /* complex[K][N] host */
  const double* q1;      /* [nb][N] host, real Lanczos start vector(s) (nb = geom.block_size) */
  double* diagG;         /* complex[K][N] host, written before the request completes */
  int* status;           /* [K] host, DYSON_ST_* flags, or NULL */
} dyson_request;

typedef struct {
  int queued, running, resident_plans, peak_running;
  size_t bytes_in_use, peak_bytes;
  uint64_t admitted, completed, plans_created, plans_evicted;
  uint64_t fused;        /* requests that ran as a segment of a fused solve */
} dyson_server_stats_t;

/* hbm_budget: most device bytes of resident plans; max_inflight: concurrent requests (1..64).
 * The server works on the device that is current at creation. */
int dyson_server_create(size_t hbm_budget, int max_inflight, dyson_server* out);
/* Finishes queued and running requests, then frees every plan and stream. */
int dyson_server_destroy(dyson_server server);
/* Queue a request; the caller keeps its buffers alive until dyson_wait returns.
 * DYSON_E_BUDGET if the request alone needs more than the budget. */
int dyson_submit(dyson_server server, const dyson_request* request, uint64_t* ticket);
/* *done = 1 once the request has finished (outputs written), else 0. */
int dyson_poll(dyson_server server, uint64_t ticket, int* done);
/* Block until the request finishes and forget the ticket.  latency_ms: submission to
 * completion; run_ms: admission to completion (each may be NULL). */
int dyson_wait(dyson_server server, uint64_t ticket, double* latency_ms, double* run_ms);
int dyson_server_stats(dyson_server server, dyson_server_stats_t* out);

/* Kernel kinds reported by dyson_profile_read. */
#define DYSON_KERNEL_INIT 0      /* start vector, per-frequency state */
#define DYSON_KERNEL_FACTOR 1    /* subdomain recursions: g_s and diag(B^-1) */
#define DYSON_KERNEL_PRECOND 2   /* interface preconditioner factors */
#define DYSON_KERNEL_XMATVEC 3   /* u = X q_j (Eqs. 6-8) */
#define DYSON_KERNEL_LANCZOS 4   /* Lanczos step, CGS2, assembly (Eq. 9) */
#define DYSON_KERNEL_FINALIZE 5  /* diag(G) to natural order */
#define DYSON_KERNEL_STATUS 6    /* per-frequency status */

/*
 * Kernel timing.  With profiling on, dyson_solve brackets every kernel it
 * launches with CUDA timing events on the stream the kernel runs on (inside
 * the captured graph they become event-record nodes).  Switching it on or
 * off drops the plan's cached graphs.  dyson_profile_read waits for the
 * device and returns, for the most recent dyson_solve, *n kernels with their
 * DYSON_KERNEL_* kind and duration in ms (at most max_kernels written).
 */
int dyson_plan_set_profiling(dyson_plan plan, int on);
int dyson_profile_read(dyson_plan plan, int max_kernels, int* kinds, float* ms, int* n);

/*
 * The same kernels as start and end times in ms from the earliest kernel start
 * of that solve (kernels of different frequency groups overlap in time), for
 * the time the GPU spends in one kind of kernel: the union of its intervals.
 * Either output may be NULL; at most max_kernels written; *n as above.
 */
int dyson_profile_spans(dyson_plan plan, int max_kernels, float* start_ms, float* end_ms, int* n);

/*
 * Work accounting of the last dyson_solve: sweeps[K][p] receives the number
 * of block forward/back substitutions (each reads the subdomain's stored
 * g_s twice) that the CTA of subdomain i performed for frequency k (summed
 * over the columns of a block plan).
 * Waits for the device.
 */
int dyson_work_counters(dyson_plan plan, int K, unsigned long long* sweeps);

/*
 * Lanczos basis of frequency k (0-based) from the last dyson_solve, for
 * checking the run step by step: Q complex[nvec][N] (host) receives q_1 ..
 * q_nvec in natural order (bilinear-normalised, Sec. 2.1), nvec <= k_max+nb
 * (block plans: column j*nb + c is column c of block j; deflated columns are 0);
 * vectors past the last step taken are left over from earlier work.  The mixed
 * form with nb = 1 and k_max <= 64 keeps its basis as double-floats (47
 * significant bits per real part); those values are widened exactly here.
 * Waits for the device; allocates a temporary device buffer.
 */
int dyson_lanczos_basis(dyson_plan plan, int k, int nvec, double* Q);

/*
 * Failure-detection self-test (the paper has no counterpart).  Every wait of
 * the solver's kernels on a copy ring is bounded by the global timer: on
 * time-out the kernel records DYSON_ST_WAIT_TIMEOUT and returns instead of
 * hanging.  This call runs that same bounded wait, on the current device, on
 * an mbarrier that nothing ever arrives on, with a limit of limit_s seconds
 * (1e-6 .. 10): *timed_out = 1 when the wait gave up and the kernel returned;
 * *waited_s (may be NULL) receives the time it waited.  The device stays
 * usable afterwards.  Synchronous; allocates 8 bytes of device memory.
 */
int dyson_wait_selftest(double limit_s, int* timed_out, double* waited_s);

/*
 * Allocation-free variant of dyson_subdomain_diag.  The paper has no
 * counterpart.  It is meant for host programs that cannot let the solver
 * allocate device memory: a simulation that reserves all of its device memory
 * in one pool at start-up and treats any later cudaMalloc as an error (the pool
 * may leave nothing free, and an allocation can stall the device while other
 * work runs), or a plugin inside another framework that owns every device
 * buffer and only lends it inputs and outputs.  No plan is needed and nothing
 * is allocated: omega [K], V [N], sigma complex[K][N] and the output diagB
 * complex[K][N] are the caller's DEVICE pointers on the current device (each is
 * checked to be device memory of that device, else DYSON_E_BAD_ARG); the work
 * is enqueued on `stream` in the FP64 form and the call returns without
 * waiting.  Slice widths up to 64 only (DYSON_E_UNSUPPORTED above); K at most
 * 65535.  Of the geometry only dim, L, t, mu, p, precision (must be
 * DYSON_FP64) and eta are read.
 *
 * All other storage lives in one fixed device array of
 * DYSON_NOALLOC_SCRATCH_BYTES that the library reserves statically: every GPU
 * that loads the library holds it until the process exits.  A geometry and K
 * that need more (index map + K x (subdomain-first diagonal + slice factors))
 * are rejected with DYSON_E_BUDGET and a message naming the bytes needed; use
 * fewer frequencies per call.  All calls share the array and it keeps the last
 * call's contents; calls whose work overlaps on the GPU (other streams or
 * threads) race on it, so callers must serialise them.  The first call on a
 * device looks up the array's device address (once per device, with that
 * device current); make that first call before any stream capture.
 */
#define DYSON_NOALLOC_SCRATCH_BYTES (32u << 20)
int dyson_subdomain_diag_noalloc(const dyson_geometry* geom, int K, const double* omega,
                                 const double* V, const double* sigma, double* diagB,
                                 void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DYSON_H */
