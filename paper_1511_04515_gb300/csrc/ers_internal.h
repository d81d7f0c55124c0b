// Internal data layout shared by the CUDA translation units of libers.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "../../include/ers.h"
#include "symbolic.h"

namespace ers {

// Piecewise-linear source value at x (constant beyond the table's ends).  The host evaluates
// the same function to decide whether a step sees a ramp, so the product and the sum are
// rounded separately on both sides (no fused multiply-add): the two agree bit for bit.
__host__ __device__ __forceinline__ double pwl_eval(const double* t, const double* v, int np,
                                                    double x) {
  if (x <= t[0]) return v[0];
  if (x >= t[np - 1]) return v[np - 1];
  int lo = 0, hi = np - 1;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (t[mid] <= x) lo = mid; else hi = mid;
  }
  const double f = (x - t[lo]) / (t[hi] - t[lo]);
#ifdef __CUDA_ARCH__
  return __dadd_rn(v[lo], __dmul_rn(f, v[hi] - v[lo]));
#else
  volatile double prod = f * (v[hi] - v[lo]);
  return v[lo] + prod;
#endif
}


// device status bits (OR-ed into ctx->d_status[0])
enum : unsigned {
  ST_SINGULAR = 1u,     // zero or tiny pivot in the refactor
  ST_NONFINITE = 2u,    // NaN/Inf met in a vector or a small dense result
  ST_TIMEOUT = 4u,      // a bounded spin-wait gave up
  ST_KRYLOV = 8u,       // exp(h H^-1) not finite
};

constexpr int MAX_M = 64;        // largest Krylov dimension supported
constexpr int MAX_RHS = 3;       // right-hand sides solved in one pass over the factors
constexpr int SPIN_LIMIT = 1 << 22;

// Per-basis device-side Arnoldi state (one per Krylov space).
struct KrylovState {
  double beta;          // ||v||
  double gv1;           // ||G v_1|| (scale of the relative residual test)
  double w0;            // ||w|| before orthogonalisation (current iteration)
  double gvnext[MAX_M + 1];
  double y[MAX_M];      // exp(h H_m^-1) e_1 of the chosen dimension
  double last;          // e_m^T H_m^-1 exp(h H_m^-1) e_1
  double res;           // last residual ratio
  double best_res;
  int built;            // Arnoldi iterations done
  int m;                // dimension chosen for the MEVP (0 = zero vector)
  int best_m;
  int done;             // 1 = converged / breakdown / zero vector: no further iterations
  int breakdown;
  int scan;             // 1 = the skipped dimensions [m_min, built] await a parallel test
  int pad[2];
};

// A set of Krylov spaces advanced in lockstep (their solves share one pass over the factors).
struct VecGroup {
  int nb;
  int slot[MAX_RHS];
  double* V[MAX_RHS];            // basis columns (stride n)
  double* H[MAX_RHS];            // (MAX_M+1) x MAX_M column-major
  const double* src[MAX_RHS];    // init: v ; mgs: solve output x (w = -x)
};

// modes of the small dense kernel
enum : int { SMALL_RESID = 0, SMALL_FINAL = 1, SMALL_FIXED_END = 2, SMALL_TEST = 3 };

// Factor and solve plan resident on the device.
struct DevicePlan {
  int n = 0, nsn = 0, nlevels = 0;
  int32_t *sn_start = nullptr, *sn_parent = nullptr, *rows = nullptr, *rel = nullptr;
  int64_t *rptr = nullptr, *d_off = nullptr, *o_off = nullptr, *front_off = nullptr;
  int32_t *lvl_sn = nullptr, *lvl_slot = nullptr, *ea_child = nullptr;
  int32_t *ch_ptr = nullptr, *ch_list = nullptr;   // children in rank order (CSR)
  int64_t* asm_dst = nullptr;
  int32_t *tile_sn = nullptr, *tile_ij = nullptr, *ptask_sn = nullptr, *ptask_r0 = nullptr;
  SolveTask *fwd = nullptr, *bwd = nullptr, *fwd_small = nullptr, *bwd_small = nullptr;
  int32_t *fwd_tgt = nullptr, *fwd_expect = nullptr, *bwd_nchunk = nullptr;
  int32_t *fwd_lane = nullptr, *bwd_lane = nullptr;   // 4 ints per lane item
  int nfwd = 0, nbwd = 0;
  // a pass whose entries are all GROUP entries: its warp tasks flattened in entry order, run
  // by self-scheduling warps (n = 0: the CTA list above is used)
  SolveTask *fwd_warp = nullptr, *bwd_warp = nullptr;
  int nfwd_warp = 0, nbwd_warp = 0;
  // factor values
  double *LDi = nullptr, *UDi = nullptr, *Lo = nullptr, *Uo = nullptr;
  double* arena = nullptr;
  // merged blocks: explicit inverses of their triangles (W x W column-major each) and the
  // first / last piece of every block
  double *ML = nullptr, *MU = nullptr;
  int32_t *grp_first = nullptr, *grp_last = nullptr;
  int ngrp = 0;
  // solve sync words: [0], [1] task counters of the two passes, then per supernode: arrivals,
  // ready / done flags, backward arrivals, forward and backward row-tile counters of merged
  // pieces, and the completed row tiles of each merged block (at its first piece)
  int32_t* sync = nullptr;   // solve_sync_words(nsn) ints
};

constexpr size_t solve_sync_words(size_t nsn) { return 2 + 6 * nsn; }

}  // namespace ers

struct ers_ctx;
namespace ers {
// shared by the translation units (defined in api.cu)
ers_status create_context(ers_ctx* c, const ers_csr* G, const ers_csr* C, const ers_csr* B,
                          const ers_mosfet* dev, int32_t ndev, const ers_pwl* u, int32_t p,
                          const ers_opts* opts);
ers_status ctx_fail(ers_ctx* c, ers_status st, const std::string& msg);
ers_status ctx_refactor(ers_ctx* c);
ers_status ctx_sync_status(ers_ctx* c);
ers_status ctx_clear_status(ers_ctx* c);
// batch.cu: a batched context on the current device
ers_status create_batch_here(ers_ctx** out, const ers_instance* inst, int32_t ninst,
                             const ers_opts* opts);

// Makes `dev` the current device for the guard's lifetime and restores the caller's device
// (dev < 0: no change).  Every public call on a context runs under one.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev)
      changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// devices.cu: a batch split over several devices (group context)
// "" if the device list is usable: ndevices >= 0, ids valid on this machine, devices != NULL
// when ndevices > 0
std::string check_device_list(const int32_t* devices, int32_t ndevices);
void lpt_partition(const double* cost, int n, int nparts, int32_t* part_of);
ers_status group_create(ers_ctx* g, const ers_instance* inst, int32_t ninst,
                        const int32_t* devices, int32_t ndevices, const ers_opts* opts);
void group_destroy(ers_ctx* g);
ers_status group_run_batch(ers_ctx* g, double t_end, double tol, int32_t max_steps,
                           int32_t* nsteps, int32_t* nreject);
ers_status group_dc(ers_ctx* g, const double* x0);
ers_status group_set_state(ers_ctx* g, double t, const double* x, double h);
ers_status group_get_state(ers_ctx* g, double* t, double* x, double* h);
ers_status group_apply(ers_ctx* g, const double* b, double* x, bool solve);
ers_status group_get_state_inst(ers_ctx* g, int32_t k, double* t, double* x, double* h);
ers_status group_records(ers_ctx* g, int32_t k, ers_step_record* out, int32_t cap,
                         int32_t* count);
ers_status group_samples(ers_ctx* g, float* X, float* T, int32_t cap, int32_t* count);
ers_status group_set_controller(ers_ctx* g, ers_mlp* mlp, int32_t parts, double margin);
ers_status group_stats(ers_ctx* g, ers_stats_t* out);
ers_status group_ctrl_stats(ers_ctx* g, int64_t* proposals, int64_t* rejected, int64_t* kv);
// f(share, index) on every share with its device current (one host thread per device)
ers_status group_call(ers_ctx* g, const std::function<ers_status(ers_ctx*, int)>& f);
}  // namespace ers

// the opaque context of the public C ABI
struct ers_ctx {
  std::string err;
  ers_opts opts{};
  int n = 0, p = 0, ndev = 0;
  ers::Symbolic sym;
  ers::DevicePlan plan;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;   // the stream the library created (destroyed with it)
  int device = 0;
  int sm_count = 0;
  int solve_ctas_per_sm = 3;           // resident CTAs per SM of the persistent solves (tunable)
  int solve_variant = 0;               // code variant of the CTA-list solve kernels (tunable)
  // all-GROUP passes: run warp-scheduled (else as the CTA list); tunable.  The defaults are
  // the faster choices on the 2000-stage chain: CTA list forward, warp-scheduled backward
  bool solve_warp_fwd = false, solve_warp_bwd = true;
  // host copies (permuted) needed by the host-side step orchestration
  std::vector<double> bp;              // sorted unique PWL corner times
  std::vector<int32_t> h_pwl_ptr;      // PWL tables (the device's copy is pwl_*)
  std::vector<double> h_pwl_t, h_pwl_v;
  std::vector<std::pair<double, double>> pwl_active;   // merged ranges where a source changes
  // device arrays (permuted node order)
  int32_t* d_perm = nullptr;                    // new -> old node index
  int32_t *G_ptr = nullptr, *G_idx = nullptr;   // union pattern of G_k
  double *Glin_val = nullptr, *G_val = nullptr; // linear values, current G_k values
  int32_t *C_ptr = nullptr, *C_idx = nullptr; double* C_val = nullptr;
  int32_t *B_ptr = nullptr, *B_idx = nullptr; double* B_val = nullptr;  // n x p
  int nnzG = 0, nnzC = 0, nnzB = 0;
  bool C_diag = false;
  double* Cdiag = nullptr;
  // PWL tables
  int32_t* pwl_ptr = nullptr; double *pwl_t = nullptr, *pwl_v = nullptr;
  double* u = nullptr;        // p
  double* slope = nullptr;    // p
  // devices (terminals already permuted; <0 = rail)
  int32_t* dev_type = nullptr; int32_t* dev_term = nullptr;  // 3 per device: d,g,s
  double* dev_par = nullptr;  // 3 per device: vt,k,lambda
  double* dev_I = nullptr;    // current at x_k
  double* dev_J = nullptr;    // 3 partials at x_k
  int32_t* stamp_ptr = nullptr; int32_t* stamp_ent = nullptr;  // per G slot: device contributions
  int32_t* node_ptr = nullptr; int32_t* node_ent = nullptr;    // per node: device incidences
  // vectors
  double *x = nullptr, *xk = nullptr, *xnew = nullptr, *F = nullptr, *rhs = nullptr;
  double *v1 = nullptr, *w1 = nullptr, *v2 = nullptr, *ve = nullptr, *tmp = nullptr;
  double* solve_buf = nullptr;       // MAX_RHS * n
  double* solve_z = nullptr;         // MAX_RHS * n: merged blocks' intermediate vectors
  double* solve_part = nullptr;      // partial sums of the merged blocks' GEMV tasks
  ers::MJob* d_mjobs = nullptr;      // inversion plan of the merged blocks
  int32_t* d_mtile = nullptr;
  double* V = nullptr;               // 3 bases, each (MAX_M+1) * n
  double* H = nullptr;               // 3 * (MAX_M+1) * MAX_M
  ers::KrylovState* ks = nullptr;    // 3
  double* red = nullptr;             // reduction scratch
  unsigned* d_status = nullptr;      // [0] status bits, [1..] barrier words
  unsigned* h_status = nullptr;      // pinned mirror
  double* h_scalars = nullptr;       // pinned scalars for host decisions
  cudaEvent_t poll_ev[4] = {};       // lagged done-flag reads of adaptive Arnoldi builds
  double* h_bpin = nullptr;          // batched: pinned per-instance reads (4 ninst doubles)
  std::vector<int32_t> h_src_inst;   // batched: instance of each PWL source
  int coop_blocks = 0;
  // state
  double t = 0.0, h = 0.0;
  bool factored = false;             // LU of G_k valid for the current x
  bool linear = true;
  bool singular_c = false;           // C has a zero row: deflate near-null eigenvalues of H_m
  ers_stats_t stats{};
  // batch: instances concatenated into one block-diagonal circuit (ninst = 1 otherwise)
  int ninst = 1;
  std::vector<int32_t> seg_off;        // ninst + 1: node ranges in the internal (permuted) order
  std::vector<int32_t> orig_off;       // ninst + 1: node ranges in the concatenated input order
  std::vector<std::vector<double>> bp_inst;
  std::vector<double> t_inst, hprop_inst;
  std::vector<int64_t> steps_inst, rejects_inst;
  int32_t* d_inst_of = nullptr;        // n: instance of each internal node
  int32_t* d_seg_off = nullptr;        // ninst + 1
  int32_t* d_src_inst = nullptr;       // p: instance of each source
  ers::KrylovState* bks = nullptr;     // 3 * ninst
  double* bH = nullptr;                // 3 * ninst * (MAX_M + 1) * MAX_M
  double *bh = nullptr, *bt = nullptr, *bred = nullptr;  // ninst each
  int32_t* bmask = nullptr;            // ninst
  int32_t* bcount = nullptr;           // 1
  unsigned long long* d_kv = nullptr;  // Krylov vectors built by the batched Arnoldi kernels
  unsigned* d_where = nullptr;         // first non-finite value of a batched run (4 words)
  double *bscan_res = nullptr, *bscan_last = nullptr, *bscan_y = nullptr;  // per (space, dim)
  // CUDA graphs of one batched Arnoldi iteration, per combination of spaces
  struct IterGraph {
    int nb = 0, ctrl = 0;
    int slot[ers::MAX_RHS] = {0, 0, 0};
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0, solves = 0, passes = 0, rhs = 0;   // per replay
  };
  std::vector<IterGraph> iter_graphs;
  bool batch_graphs = true;
  int32_t* bj = nullptr;               // device index of the current Arnoldi iteration
  int32_t* bscan_fin = nullptr;
  std::vector<int32_t> scan_mask;      // instances masked in the current batch_bases call
  int ctrl_parts = 0;                  // ERS_CTRL_H | ERS_CTRL_M: which proposals are used
  double ctrl_margin = 0.0;            // log2 margin subtracted from proposed step ratios
  // learned step controller of batched runs
  ers_mlp* ctrl = nullptr;             // not owned; nullptr = plain controller
  bool trace = false;                  // keep every record (else the last ERS_CTRL_HISTORY)
  std::vector<std::vector<ers_step_record>> recs;   // per instance, accepted steps
  std::vector<int32_t> mstart_inst;    // first dimension of the residual test per instance
  std::vector<uint8_t> proposed_inst;  // next step of the instance is a network proposal
  int64_t ctrl_proposals = 0, ctrl_rejected = 0;
  int32_t* d_mstart = nullptr;         // ninst
  int32_t* d_mused = nullptr;          // ninst
  double* bdf = nullptr;               // ninst
  float *d_feat = nullptr, *d_pred = nullptr;   // ninst x 32, ninst x 2
  // a batch over several devices (ers_create_batch with ndevices > 1): the per-device batched
  // contexts; this context holds no device memory and only dispatches
  std::vector<ers_ctx*> group;
  std::vector<int32_t> group_dev;                 // device of each share
  std::vector<std::vector<int32_t>> group_inst;   // input-order instances of each share
  std::vector<int32_t> inst_grp, inst_loc;        // share and local index of each instance
  std::vector<int32_t> inst_n, inst_off;          // node count / offset of each instance
  std::vector<ers_mlp*> group_nets;               // network copies, one per share (owned)
  bool grouped = false;                           // set by group_create, even on failure
  bool is_group() const { return grouped; }
  // profiling of the solve kernels (CUDA events on the context's stream)
  bool profile = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_free, ev_used;
};
