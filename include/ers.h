/*
 * ers.h -- C ABI of a GB300 (sm_103a) FP64 implementation of the exponential
 * Rosenbrock-Euler (ER) circuit transient with the invert-Krylov matrix exponential
 * (Zhuang, Yu, Kang, Wang, Cheng, DAC 2015, arXiv 1511.04515).
 *
 * Problem (Sec. II, Eq. 1; Sec. III linearised form):
 *     C x'(t) + G_lin x + i_dev(x) = B u(t)
 * x: node voltages (n), C: capacitances (n x n), G_lin: linear conductances (n x n),
 * i_dev: square-law MOSFET currents, B (n x p) with piecewise-linear inputs u(t).
 * At x_k the step uses G_k = G_lin + d i_dev/dx (x_k) and the remainder
 * F(x) = (G_k - G_lin) x - i_dev(x), so that C x' = -G_k x + F(x) + B u (Sec. III).
 *
 * Conventions shared by every entry point:
 *  - All pointers are HOST pointers unless a name ends in _dev.  Inputs are copied; the
 *    caller keeps ownership of everything it passes and of every output buffer.
 *  - CSR matrices are 0-based with sorted, unique column indices per row.
 *  - Every call returns an ers_status and never aborts the process; on failure
 *    ers_last_error() returns a message.  No call traps or hangs the GPU: device-side
 *    waits are bounded and report ERS_ERR_TIMEOUT.
 *  - A context is bound to one CUDA device (the first entry of the device list given at
 *    creation, or the device current then) and to one CUDA stream (ers_set_stream).  Every
 *    call makes the context's device current for its duration and restores the caller's
 *    current device before returning.  Calls on one context must not overlap.
 */
#ifndef ERS_H
#define ERS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ers_ctx ers_ctx;

typedef enum {
  ERS_OK = 0,
  ERS_ERR_INVALID = 1,          /* bad argument, bad CSR, step crossing a PWL corner   */
  ERS_ERR_SINGULAR = 2,         /* zero / tiny pivot in the static-pivot LU of G_k      */
  ERS_ERR_NONFINITE = 3,        /* NaN or Inf in inputs or results                       */
  ERS_ERR_STEP_UNDERFLOW = 4,   /* adaptive h fell below h_min                           */
  ERS_ERR_KRYLOV = 5,           /* exp(h H_m^{-1}) e_1 not finite at any usable dimension */
  ERS_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up                    */
  ERS_ERR_CUDA = 7,             /* CUDA runtime error                                    */
  ERS_ERR_OOM = 8               /* device allocation failed                              */
} ers_status;

typedef struct {
  int32_t n_rows, n_cols, nnz;
  const int32_t* rowptr;        /* n_rows + 1 */
  const int32_t* colidx;        /* nnz */
  const double* val;            /* nnz */
} ers_csr;

/* MOSFET record (square-law stand-in for the paper's BSIM3 devices, Sec. V).
 * type 0 = NMOS, 1 = PMOS; terminals are node indices, -1 = ground, -2 = vdd rail.
 * Current flows d -> s; source/drain swap when v_ds < 0; PMOS mirrors NMOS. */
typedef struct {
  int32_t type, d, g, s;
  double vt, k, lambda;
} ers_mosfet;

/* Piecewise-linear input (Sec. III, u linear on every step): npts corner times
 * (strictly increasing) and values; constant before the first and after the last. */
typedef struct {
  int32_t npts;
  const double* t;
  const double* v;
} ers_pwl;

typedef struct {
  double eps_krylov;   /* Krylov residual tolerance of Eq. 16, relative (default 1e-7, Sec. V) */
  double E_rr;         /* absolute error budget of Alg. 2 (0: tol * max(1, ||x||_inf))          */
  double alpha;        /* h <- alpha h on rejection (Alg. 2, default 0.5)                        */
  double beta;         /* h <- beta h after a fast acceptance (Alg. 2, default 2)                */
  double gamma;        /* ER-C correction weight (Eq. 17, default 0.1)                            */
  double h_min;        /* step underflow limit (default 1e-20 s)                                  */
  double h_max;        /* largest step (0: t_end / 100)                                           */
  double h_init;       /* first step (0: h_max)                                                   */
  double vdd;          /* supply rail voltage for terminals tagged -2 (default 1 V)               */
  double gmin;         /* conductance added from every node to ground (default 0: the netlist
                          carries its own; a MOSFET stage needs some, see the inverter chains) */
  int32_t i_grow;      /* grow h when the retry count i < i_grow (Alg. 2, default 5)              */
  int32_t m_min;       /* first dimension at which Eq. 16 is tested (default 3)                   */
  int32_t m_max;       /* Algorithm 1's m_c (default 40, at most 64)                              */
  int32_t combined_vector; /* 1: one Krylov space on v1 + v2 instead of two (default 0)           */
  int32_t correction;  /* 1: ER-C (Eq. 20), 0: ER (default 0)                                      */
  int32_t ordering;    /* fill-reducing ordering of G_k's pattern (default 1):
                          0: nested dissection, separator = the BFS level at the median;
                          1: the smallest BFS level leaving >= 35% of the part on each side,
                             from either end of the pseudo-diameter (less fill on meshes) */
} ers_opts;

typedef struct {
  int64_t steps;               /* accepted steps (a batched context: rounds)            */
  int64_t rejects;             /* rejected tries                                         */
  int64_t refactors;           /* LU refactors of G_k                                    */
  int64_t krylov_vectors;      /* Arnoldi directions built (every space, every instance) */
  int64_t solves;              /* right-hand sides through the L and U solves            */
  int32_t n, nsn, nlevels, etree_height, max_front;   /* symbolic analysis              */
  int64_t nnz_L, factor_doubles, arena_doubles;
  double refactor_flops;
  int64_t kernel_launches;     /* kernels launched by the library so far              */
  int64_t solve_passes;        /* forward+backward solve pairs (any number of RHS)    */
  int64_t solve_rhs;           /* right-hand sides solved                              */
  double solve_ms;             /* device time of the solve kernels (profiling on; solves
                                  replayed inside CUDA graphs are not timed)           */
  double solve_bytes_per_pass; /* factor bytes one solve pair reads (values+indices)  */
  double solve_fma_per_rhs;    /* FP64 FMAs of one solve pair per right-hand side     */
  int64_t graph_launches;      /* CUDA graph launches (batched Arnoldi iterations)     */
  int64_t merged_blocks;       /* dense separator triangles solved through their inverse */
  int64_t merged_columns;      /* columns in those blocks                               */
  int64_t merged_inverse_doubles; /* doubles of the two inverses (M_L and M_U)          */
  double merged_inverse_flops; /* flops of computing the inverses after each refactor   */
  int64_t host_syncs;          /* stream synchronisations of the stepping calls (the host
                                  waits for the device queue to drain)                   */
  int64_t host_polls;          /* lagged reads of the Krylov spaces' done flags: the host
                                  waits for an event two iterations back while the
                                  device runs the iteration queued after it             */
} ers_stats_t;

/* One circuit of a batch (ers_create_batch): the same data ers_create takes. */
typedef struct {
  const ers_csr* G;            /* n x n linear conductances */
  const ers_csr* C;            /* n x n capacitances        */
  const ers_csr* B;            /* n x p source incidence    */
  const ers_mosfet* dev;       /* ndev devices (may be NULL if ndev = 0) */
  int32_t ndev;
  const ers_pwl* u;            /* p PWL inputs */
  int32_t p;
} ers_instance;

/* Fill opts with the defaults listed above. */
ers_status ers_default_opts(ers_opts* opts);

/* Create a simulation context (Alg. 2 "initialization phase": load netlist, build linear
 * matrices; Sec. II problem statement C x' + G x + i(x) = B u).  G_lin, C: n x n; B: n x p;
 * dev: ndev MOSFETs (may be NULL if ndev = 0); u: p PWL inputs.  devices / ndevices: the
 * CUDA device list; ndevices = 0 (devices may be NULL) uses the current device, 1 uses
 * devices[0]; a single circuit does not shard (every G_k^-1 of Algorithm 1 couples all of its
 * nodes), so ndevices > 1 is ERS_ERR_INVALID -- create one context per device for replicas.
 * A device id that does not exist is ERS_ERR_INVALID.  Performs the one-time symbolic
 * analysis of G_k's pattern (the union of G_lin and the device stamps) and allocates device
 * memory.  The state starts at t = 0, x = 0; call ers_dc for the DC operating point.
 * opts may be NULL (defaults).
 * Every node needs a capacitance (a nonzero entry in its row of C): a node without one
 * makes C singular and H_m of Eq. 14 singular with it, which the small dense stage does not
 * handle; such a C is refused with ERS_ERR_INVALID before any device work. */
ers_status ers_create(ers_ctx** out, const ers_csr* G_lin, const ers_csr* C, const ers_csr* B,
                      const ers_mosfet* dev, int32_t ndev, const ers_pwl* u, int32_t p,
                      const int32_t* devices, int32_t ndevices, const ers_opts* opts);

/* Batched context over ninst independent circuits (Monte Carlo corners, parameter sweeps;
 * the paper simulates one circuit at a time).  The instances are concatenated into one
 * block-diagonal circuit: one symbolic analysis, one refactor and one solve pass per step
 * cover all of them, while Algorithm 1 and 2 run per instance (own Krylov spaces and
 * dimensions, step sizes, times, PWL corners and error tests).  State access: ers_dc,
 * ers_set_state / ers_get_state act on the concatenated vector (instance k's nodes follow
 * instance k-1's); ers_get_state_inst reads one instance.
 * devices / ndevices: the CUDA device list (0 = the current device).  With ndevices > 1 the
 * instances are split over the listed devices by longest-processing-time-first
 * (ers_partition_lpt) on the estimated cost nnz(G_lin) + n + 6 ndev of each instance, with no
 * exchange between devices on the data path: each share is a batched context of its own on
 * its device, shares on different devices run concurrently (one host thread per device),
 * shares listed on the same device one after the other, and every call gathers per-instance
 * results on the host in input order.  Such a context refuses ers_set_stream, ers_mevp,
 * ers_solve_dev_noalloc and the _dev state calls (ERS_ERR_INVALID); ers_stats adds the
 * shares' counters (steps: the largest share's rounds); a network given to
 * ers_batch_set_controller is copied once per share. */
ers_status ers_create_batch(ers_ctx** out, const ers_instance* inst, int32_t ninst,
                            const int32_t* devices, int32_t ndevices, const ers_opts* opts);
/* (opts->correction and opts->combined_vector are single-context options: ERS_ERR_INVALID
 * here.  ers_step / ers_run on a batched context return ERS_ERR_INVALID: it steps with
 * ers_run_batch.) */

/* Advance every instance of a batched context to t_end with Algorithm 2 (at most max_steps
 * rounds when max_steps > 0; in a round every unfinished instance takes one accepted step).
 * nsteps / nreject (ninst entries each, may be NULL) receive the per-instance counts of
 * accepted and rejected steps of this call.  ers_set_state / ers_set_state_dev on a batched
 * context set every instance's time and proposed step and start a new step history (the
 * learned controller's records and pending proposals are cleared). */
ers_status ers_run_batch(ers_ctx* ctx, double t_end, double tol, int32_t max_steps,
                         int32_t* nsteps, int32_t* nreject);

/* Time, state (n_k doubles, the instance's own node order) and proposed step of instance k. */
ers_status ers_get_state_inst(const ers_ctx* ctx, int32_t k, double* t, double* x, double* h);

/* ---- Learned step controller (the paper's controller is the plain rule of Alg. 2: reject ->
 * h = alpha h with the same Krylov spaces, accept -> h = beta h while the step saw fewer than
 * i_grow rejections).  The learned form keeps the error test of Eq. 15 as the arbiter: a network
 * proposes the next (h, m) of each instance from its last 8 accepted steps; a rejected
 * proposal falls back to the plain rule (h = alpha h, same spaces).  The proposed m is the
 * Krylov dimension from which the residual test of Eq. 16 is evaluated; the basis still grows
 * until that test passes, so a proposal changes cost, never the accuracy bar. ---- */

/* One accepted step of one instance. */
typedef struct {
  double h;        /* accepted step size */
  double h_max;    /* step-size cap of the run */
  double err;      /* ||e_rr||_inf of the accepted step (Eq. 15) */
  double E;        /* error budget E_rr of the step */
  double dF;       /* ||F(x_{k+1}) - F(x_k) - J_k (x_{k+1} - x_k)||_inf (0 for linear circuits) */
  int32_t m;       /* largest Krylov dimension used by the step's solution spaces */
  int32_t m_max;   /* dimension cap of the run */
  int32_t landed;  /* 1 = h was cut to land on a PWL corner or t_end */
  int32_t retries; /* rejections before acceptance */
} ers_step_record;

#define ERS_CTRL_HISTORY 8     /* accepted steps the network sees */
#define ERS_CTRL_FEATURES 32   /* 4 features per step */

/* Features of the network input from the last min(count, 8) records (recs[count-1] is the
 * latest; missing older steps repeat the oldest one).  For step j back (j = 0 latest):
 *   f[4j+0] = clamp(log10(h / h_max), -6, 0) / 3
 *   f[4j+1] = m / m_max
 *   f[4j+2] = clamp(log10(err / E), -6, 1) / 3        (err = 0 reads as -6)
 *   f[4j+3] = (clamp(log10 dF, -12, 0) + 6) / 6       (dF = 0 reads as -12)
 * Host-only; count >= 1. */
ers_status ers_ctrl_features(const ers_step_record* recs, int32_t count, float* out);

/* Training target of the step after recs[count-1] given the next record `next`:
 *   t[0] = clamp(log2(next.h / h_k) + log2(clamp(0.8 sqrt(next.E / next.err), 1, 2)), -3, 2)
 *          (the step the plain controller accepted, widened by the headroom its error left)
 *   t[1] = next.m / next.m_max
 * Returns ERS_ERR_INVALID for a `next` that landed on a corner (its h says nothing about the
 * error).  Host-only. */
ers_status ers_ctrl_target(const ers_step_record* recs, int32_t count, const ers_step_record* next,
                           float* t);

/* Next step from a network output y (2 floats) and the last accepted step `last`:
 *   l = clamp(y[0] - margin, -3, 2)   (non-finite y[0]: l = 1)
 *   r = clamp(-log2(last.err / last.E) / 2, -3, 6)   (err = 0: r = 6), the log2 of the ratio
 *       that lands on the budget under the local error model err ~ h^2
 *   l = clamp(l, min(0, r - 1), max(0, r + 1))   (a safety band around the network)
 *   h_next = min(last.h 2^l, last.h_max)
 *   m_start = clamp(round(y[1] last.m_max) - 1, m_min, last.m_max)   (non-finite: m_min)
 * Host-only. */
ers_status ers_ctrl_propose(const float* y, const ers_step_record* last, double margin,
                            int32_t m_min, double* h_next, int32_t* m_start);

/* Network of the learned controller: 32 -> 64 -> 64 -> 64 -> 2, ReLU, BF16 weights and
 * activations with FP32 accumulation on the tensor cores, FP32 master weights, Adam.
 * Parameter vector (FP32, ers_mlp_nparam() entries): W1 (64x32 row-major), b1, W2 (64x64),
 * b2, W3 (64x64), b3, W4 (2x64), b4.  Outputs: y[0] = log2(h_next / h_k), y[1] = m_next/m_max. */
typedef struct ers_mlp ers_mlp;
/* Number of parameters (10,562). */
int32_t ers_mlp_nparam(void);
/* He-initialised weights (seeded), zero biases, zero Adam moments. */
ers_status ers_mlp_create(ers_mlp** out, uint64_t seed);
/* Copy ers_mlp_nparam() FP32 parameters in (the BF16 copy is refreshed; Adam moments are
 * kept) or out (host buffers, caller-owned). */
ers_status ers_mlp_set_params(ers_mlp* mlp, const float* params);
ers_status ers_mlp_get_params(const ers_mlp* mlp, float* params);
/* Y (n x 2) = network(X (n x 32)); host buffers, row-major. */
ers_status ers_mlp_forward(ers_mlp* mlp, const float* X, int32_t n, float* Y);
/* Same with device buffers, enqueued on `stream` (a cudaStream_t; NULL = the network's own). */
ers_status ers_mlp_forward_dev(ers_mlp* mlp, const float* X_dev, int32_t n, float* Y_dev,
                               void* stream);
/* Gradient (ers_mlp_nparam() floats, may be NULL) and value of the loss
 * L = (1/n) sum_s ||y_s - T_s||^2 over the n samples (host buffers). */
ers_status ers_mlp_grad(ers_mlp* mlp, const float* X, const float* T, int32_t n, float* grad,
                        float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the gradient of L over
 * the n samples; loss receives L before the step. */
ers_status ers_mlp_adam_step(ers_mlp* mlp, const float* X, const float* T, int32_t n, float lr,
                             float* loss);
/* `epochs` passes over the n samples in a seeded random order, one Adam step per minibatch of
 * `batch` samples; final_loss = L of the last minibatch before its step. */
ers_status ers_mlp_train(ers_mlp* mlp, const float* X, const float* T, int32_t n, int32_t epochs,
                         int32_t batch, float lr, uint64_t seed, float* final_loss);
/* Text of the network's last failure (owned by the network; "" when none, "null" for a NULL
 * network). */
const char* ers_mlp_last_error(const ers_mlp* mlp);
/* Free the network and its device memory; NULL is ignored. */
void ers_mlp_destroy(ers_mlp* mlp);

/* Use `mlp` (not owned; must outlive the runs, NULL = plain controller) as the step proposer of
 * a batched context.  parts selects which proposals are used: ERS_CTRL_H (the next step size;
 * otherwise the plain rule's), ERS_CTRL_M (the first dimension of the residual test; otherwise
 * m_min), or both.  margin >= 0 (log2 units) is subtracted from every proposed step ratio:
 * h_next = h_k 2^(y0 - margin).  In a batch one rejected instance makes the whole round
 * repeat its error basis, so a batch wants fewer rejections than a single circuit does. */
#define ERS_CTRL_H 1
#define ERS_CTRL_M 2
ers_status ers_batch_set_controller(ers_ctx* ctx, ers_mlp* mlp, int32_t parts, double margin);
/* Keep every accepted step's record (enable = 1) instead of the last 8; clears the records. */
ers_status ers_batch_trace(ers_ctx* ctx, int32_t enable);
/* Records of instance k: *count receives how many are kept; up to cap are copied to out. */
ers_status ers_batch_records(const ers_ctx* ctx, int32_t k, ers_step_record* out, int32_t cap,
                             int32_t* count);
/* Training samples from the kept records of every instance: one per accepted step k whose
 * successor did not land on a corner (features of steps <= k, target from step k+1).  X: cap x
 * 32, T: cap x 2 (may be NULL to count); *count receives the number of samples available. */
ers_status ers_batch_samples(const ers_ctx* ctx, float* X, float* T, int32_t cap, int32_t* count);
/* Batched Arnoldi iterations as CUDA graphs (enable = 1, the default) or as separate launches.
 * One graph per combination of Krylov spaces (the solution spaces, the error space) holds an
 * iteration: C v_j, the forward and backward solves, Gram-Schmidt and the dimension test; the
 * iteration index lives on the device, so the same graph is replayed for every j.  Graphs are
 * captured on the context's stream; on the legacy default stream (which cannot be captured)
 * or if a capture fails, the context falls back to separate launches. */
ers_status ers_batch_set_graphs(ers_ctx* ctx, int32_t enable);

/* Controller counters of the batched runs so far: proposals made by the network, proposals
 * rejected by the error test (each falls back to the plain rule), Krylov vectors built. */
ers_status ers_batch_ctrl_stats(const ers_ctx* ctx, int64_t* proposals, int64_t* rejected,
                                int64_t* krylov_vectors);

/* Bind the context to a CUDA stream (cudaStream_t passed as void*; NULL = the private stream
 * created at ers_create).  All device work of later calls is ordered on it.  The caller keeps
 * ownership of its stream, which must outlive the context's use of it; ers_destroy destroys
 * only the private stream. */
ers_status ers_set_stream(ers_ctx* ctx, void* stream);

/* x(0) = DC solution (Alg. 2): Newton on G_lin x + i_dev(x) = B u(0) through the same LU
 * kernels (voltage step clamp 0.5 V, at most 50 iterations, residual 1e-12 A).
 * x0_guess (n, may be NULL = zeros) is the starting point.  A long chain of gates needs a
 * guess near its logic levels (a nodeset): linearised at 0 V every stage is an amplifier
 * (gain gm/gds ~ 30 in saturation) and the Newton system of k stages grows like gain^k until
 * it overflows, which shows as ERS_ERR_SINGULAR or ERS_ERR_NONFINITE.  Sets t = 0. */
ers_status ers_dc(ers_ctx* ctx, const double* x0_guess);

/* Device evaluation at the current x, stamping of G_k and the numeric LU refactor of G_k
 * (Alg. 2: "Derive C_k, G_k, F_k" and "LU_decompose(G_k)"; C is never factored). */
ers_status ers_refactor(ers_ctx* ctx);

/* One ER (ER-C if opts.correction) step of exactly h from the current (t, x) (Eq. 13;
 * error Eq. 15/19; correction Eq. 20).  m > 0: every Krylov space uses exactly m Arnoldi
 * iterations (fewer only at a happy breakdown); m = 0: the dimension is chosen by the
 * residual test of Eq. 16 (Algorithm 1).  [t, t+h] must not contain a PWL corner
 * (ERS_ERR_INVALID).  Refactors G_k if x changed since the last factorisation.  On
 * success x <- x_{k+1}, t <- t + h.  m_used (may be NULL) receives the dimension of the
 * first Krylov space; err_inf (may be NULL) receives ||e_rr||_inf (0 for linear circuits). */
ers_status ers_step(ers_ctx* ctx, double h, int32_t m, int32_t* m_used, double* err_inf);

/* Adaptive transient from the current state to t_end (Alg. 2): one LU per accepted step,
 * rejected tries shrink h by alpha and reuse the solution's Krylov bases (no LU); tol
 * sets E_rr = tol * max(1 V, ||x_k||_inf) unless opts.E_rr > 0.  Steps are clipped to
 * PWL corners, h_max and t_end.  max_steps > 0 stops after that many accepted steps
 * (the proposed h is kept in the context, so a later call continues seamlessly). */
ers_status ers_run(ers_ctx* ctx, double t_end, double tol, int32_t max_steps, int32_t* nsteps,
                   int32_t* nreject);

/* State access (original node order; caller-owned buffers of n doubles). */
ers_status ers_get_state(const ers_ctx* ctx, double* t, double* x, double* h);
ers_status ers_set_state(ers_ctx* ctx, double t, const double* x, double h);
/* Same on device buffers (n doubles, original node order) for callers whose data already
 * lives in GPU memory; ordered on the context's stream. */
ers_status ers_get_state_dev(const ers_ctx* ctx, double* x_dev);
ers_status ers_set_state_dev(ers_ctx* ctx, double t, const double* x_dev, double h);

/* Building blocks, exposed for verification of each stage against an independent CPU
 * implementation.  Vectors are host buffers of n doubles in original node order. */
/* x = G_k^{-1} b with the current factorisation (forward + backward supernodal solves). */
ers_status ers_solve(ers_ctx* ctx, const double* b, double* x);
/* y = C v (sparse matrix-vector product with the capacitance matrix). */
ers_status ers_spmv_C(ers_ctx* ctx, const double* v, double* y);
/* MEVP_IKS (Algorithm 1): out = ||v|| V_m exp(h H_m^{-1}) e_1 with the current G_k; m > 0
 * fixed dimension, m = 0 adaptive by Eq. 16.  m_used may be NULL. */
ers_status ers_mevp(ers_ctx* ctx, const double* v, double h, int32_t m, double* out,
                    int32_t* m_used);
/* Small dense stage (Eq. 14, Eq. 16): for the m x m upper-left block of H (column-major,
 * leading dimension ldh), y = exp(h H^{-1}) e_1 (m doubles) and
 * last = e_m^T H^{-1} exp(h H^{-1}) e_1.  Runs the same device kernel the step uses. */
ers_status ers_phi_small(ers_ctx* ctx, const double* H, int32_t ldh, int32_t m, double h,
                         double* y, double* last);

/* Allocation-free solve, x_dev = G_k^{-1} b_dev (n doubles each, device memory of the
 * context's device, original node order).  The paper has no counterpart: this exists for
 * callers that may not allocate device memory at the point where they solve -- code whose
 * device memory is owned by a framework's pool allocator (memory the pool did not hand out
 * breaks its accounting), and latency-bound loops that forbid allocator calls (cudaMalloc
 * and cudaFree can synchronise the device and take unbounded time).  It calls no
 * cudaMalloc/cudaFree: the solve kernels' scratch (dependency counters) is a fixed 12 MiB
 * static device array of the library, shared by every call on a device and held by every
 * GPU that loads the library until exit.  Limits and rules: contexts whose factor has more
 * than 524288 supernodes are rejected with ERS_ERR_INVALID; the context must hold a
 * factorisation (ers_refactor, ers_dc or a step first, else ERS_ERR_INVALID); b_dev and
 * x_dev must be device (or managed) memory of the context's device, anything else is
 * ERS_ERR_INVALID before any kernel runs; calls whose solves overlap on the GPU (on any
 * context of the same device) race on the shared scratch.  The first call on a device
 * looks up the array's device address and keeps it for the life of the process (a
 * cudaDeviceReset invalidates it).  Uses the context's stream and its internal work vector;
 * the call waits for the stream before returning (it synchronises, so it cannot be made
 * while the stream is being captured into a CUDA graph).  The caller's current device is
 * restored on return. */
ers_status ers_solve_dev_noalloc(ers_ctx* ctx, const double* b_dev, double* x_dev);

/* Failure-path self-test: a kernel waits, with the bounded wait every device-side dependency
 * uses, on a flag that nothing sets.  Returns ERS_ERR_TIMEOUT (the wait gave up after its
 * poll limit, under a second, and recorded the timeout instead of hanging); the context's
 * status is cleared again and the context stays usable. */
ers_status ers_wait_selftest(ers_ctx* ctx);

/* Autotuner of the persistent triangular-solve kernels: with the current factor of G_k (the
 * context refactors first if needed) time `passes` solve passes of `nrhs` (1-3) right-hand
 * sides for 1, 2 and 3 resident CTAs per SM (any count is deadlock-free: a task only waits on
 * earlier tasks of the ordered work list), each in both code variants of the CTA-list solve
 * kernels (their register allocations differ; which is faster depends on the factor) and,
 * where a pass's work list holds only small-supernode groups, with that pass run from the CTA
 * list or warp-scheduled; keep the fastest combination for the context's later solves.  ms (3 doubles, may be NULL)
 * receives the average pass time of each count (its faster variant); *chosen (may be NULL)
 * the count kept.  Changes no result: the same tasks run with the same dependencies. */
ers_status ers_autotune(ers_ctx* ctx, int32_t nrhs, int32_t passes, double* ms, int32_t* chosen);

/* Host-only check of the refactor plan and the triangular-solve work lists built for a
 * pattern (no GPU).  Refactor: fronts whose lives overlap occupy disjoint arena ranges, every
 * front and assembly target lies inside the arena, no two entries of A assemble into one
 * position, and every relative index of a child's rows points inside its parent's front.
 * Solves: every supernode is computed by exactly one task per direction, the row chunks of a
 * large supernode cover its rows exactly once, every forward unit arrives at exactly the
 * supernodes owning the rows it updates, every backward unit waits for the nearest owner of
 * the rows it reads, and every wait of a task refers to an earlier entry of its list (the
 * property that makes the persistent solves deadlock-free).
 * counts (8 values, may be NULL): forward and backward CTA entries, lane items (fwd, bwd),
 * warp-task supernodes (fwd, bwd), supernodes solved by whole CTAs (fwd, bwd: DIAG entries
 * and the pieces of merged blocks, the dense separator triangles solved through their
 * explicit inverse).  Merged blocks are also checked: their pieces nest into one triangle,
 * every row tile's GEMV tasks cover its columns once and come after the arrivals (forward)
 * or far chunks (backward) they read, and every inversion job stays inside its arrays.  ERS_ERR_INVALID with a
 * violated property (or a malformed pattern).  opts (may be NULL: defaults) selects the
 * ordering, as in ers_create. */
ers_status ers_solve_plan_check(const ers_csr* pattern, const ers_opts* opts, int64_t* counts);

/* Host-only export of one array of the symbolic plan built for a pattern (no GPU), for
 * checking the plan outside the library.  which selects the array; int32 arrays: PERM
 * (new -> old), SN_START (nsn+1), SN_PARENT, LEVEL, ROWS (off-diagonal rows of each
 * supernode, new order), REL (their positions in the parent's front), A_PTR, A_IDX (the
 * pattern in the new order), A_SRC (each new slot's index in the given CSR), CH_PTR, CH_LIST
 * (children of each supernode in extend-add order), LVL_SLOT_PTR, LVL_SLOT (slots by level);
 * int64 arrays: RPTR (nsn+1), FRONT_OFF (arena offset of each f x f column-major front,
 * f = width + rows), ASM_DST (arena position of each slot), ARENA (one value: the arena size).
 * With out == NULL only *len (the element count) is set; otherwise out receives *len
 * elements of the array's type.  ERS_ERR_INVALID for an unknown which or a malformed pattern. */
enum { ERS_PLAN_PERM = 0, ERS_PLAN_SN_START, ERS_PLAN_SN_PARENT, ERS_PLAN_LEVEL, ERS_PLAN_ROWS,
       ERS_PLAN_REL, ERS_PLAN_A_PTR, ERS_PLAN_A_IDX, ERS_PLAN_A_SRC, ERS_PLAN_CH_PTR,
       ERS_PLAN_CH_LIST, ERS_PLAN_LVL_SLOT_PTR, ERS_PLAN_LVL_SLOT, ERS_PLAN_RPTR,
       ERS_PLAN_FRONT_OFF, ERS_PLAN_ASM_DST, ERS_PLAN_ARENA };
ers_status ers_plan_array(const ers_csr* pattern, const ers_opts* opts, int32_t which, void* out,
                          int64_t* len);

/* Host-only: the ramp test of a step's set-up (Eq. 12-13: the v2 and w1 terms exist only when
 * some input has a non-zero slope (u(t + h) - u(t)) / h over the step).  *ramp = 1 when some
 * of the p PWL inputs gives pwl(t + h) != pwl(t), evaluated with the device kernel's
 * arithmetic (product and sum rounded separately, so the two decisions agree bit for bit);
 * ers_step and ers_run take this decision on the host instead of reading the slopes back.
 * ERS_ERR_INVALID for a NULL pointer or corner times that do not increase. */
ers_status ers_pwl_ramp(const ers_pwl* u, int32_t p, double t, double h, int32_t* ramp);

/* Host-only: longest-processing-time-first partition of n jobs with costs cost[i] >= 0 over
 * nparts >= 1 parts (the device split of ers_create_batch): jobs by decreasing cost (ties:
 * lower index first) each onto the least-loaded part (ties: lower part), which keeps the
 * largest load within (4/3 - 1/(3 nparts)) of the optimum (Graham 1969).  part_of receives
 * n part numbers.  ERS_ERR_INVALID for a negative or non-finite cost. */
ers_status ers_partition_lpt(const double* cost, int32_t n, int32_t nparts, int32_t* part_of);

/* Measured FP64 FMA rate of a device, the roofline denominator of the FP64 solves (not in the
 * paper; GB300 issues FP64 at 1/64 of its FP32 rate, so the supernodal solves, one FMA per
 * 8-byte factor value, are bound by it rather than by HBM).  Times a kernel of 8 independent
 * FMA chains per thread on 8 CTAs of 256 threads per SM with CUDA events, best of 5 after a
 * warm-up launch; *tflops receives 2 x FMAs / time.  ERS_ERR_INVALID for a device that does
 * not exist. */
ers_status ers_fp64_fma_peak(int32_t device, double* tflops);

/* Statistics and symbolic-analysis figures.  Synchronises the context's stream. */
ers_status ers_stats(const ers_ctx* ctx, ers_stats_t* out);
/* Turn CUDA-event timing of the triangular-solve kernels on (1) or off (0); resets the
 * accumulated solve_ms.  Events are recorded on the context's stream around each solve. */
ers_status ers_profile(ers_ctx* ctx, int32_t enable);

/* Host-only symbolic analysis of an n x n pattern (no GPU needed): fills the fields of
 * out that describe the ordering and factor (n, nsn, nlevels, etree_height, max_front,
 * nnz_L, factor_doubles, arena_doubles, refactor_flops).  perm (may be NULL) receives the
 * fill-reducing permutation new -> old.  opts (may be NULL: defaults) selects the ordering,
 * as in ers_create. */
ers_status ers_analyze(const ers_csr* pattern, const ers_opts* opts, ers_stats_t* out,
                       int32_t* perm);

/* Text of the context's last failure (owned by the context, valid until its next call). */
const char* ers_last_error(const ers_ctx* ctx);
/* Free the context and all its device memory; a stream set by the caller is left alone. */
void ers_destroy(ers_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ERS_H */
