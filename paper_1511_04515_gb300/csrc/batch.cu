// Batched ER transient: many independent circuit instances (Monte Carlo corners, parameter
// sweeps) in one context.  The instances are concatenated into one block-diagonal circuit, so
// the device evaluation, the refactor of G_k (Alg. 2) and every supernodal solve pass cover
// all instances in one launch each.  Everything that Algorithm 1 and 2 decide per circuit is
// per instance: inner products and norms are segmented (the nested-dissection order keeps an
// instance's nodes contiguous), every instance has its own Krylov spaces, dimension, step size,
// time, PWL corners and error test.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "controller.h"
#include "ers_internal.h"
#include "kcommon.cuh"
#include "kdense.cuh"

namespace ers {

void launch_dev_eval(ers_ctx* c, const double* x, double* dev_I, int with_jac);
void launch_node_F(ers_ctx* c, int mode, const double* dev_In, const double* xn, double* out);
cudaError_t launch_solve(ers_ctx* c, double* y, int nrhs);
cudaError_t launch_solve_skip(ers_ctx* c, double* y, int nrhs, const int* const* done, int ndone);
void launch_spmv(ers_ctx* c, const int32_t* ptr, const int32_t* idx, const double* val,
                 const double* x, double* y, double alpha);

constexpr int BT = 512;   // threads of the per-instance kernels

// per source: u = u(t_inst), slope = (u(t_inst + h_inst) - u) / h_inst (0 for idle instances)
__global__ void k_bpwl(int p, const int32_t* ptr, const double* tt, const double* vv,
                       const int32_t* src_inst, const double* t_arr, const double* h_arr,
                       const int32_t* mask, double* u, double* slope) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p) return;
  int i = src_inst[q];
  int o = ptr[q], np = ptr[q + 1] - ptr[q];
  double t = t_arr[i], h = h_arr[i];
  double u0 = pwl_eval(tt + o, vv + o, np, t);
  u[q] = u0;
  slope[q] = (mask[i] && h > 0.0) ? (pwl_eval(tt + o, vv + o, np, t + h) - u0) / h : 0.0;
}

struct BArgs {
  int n, ninst, nb, j, adaptive, mode;
  int slot[MAX_RHS];
  double* V[MAX_RHS];
  double* src[MAX_RHS];        // init: v ; mgs: solve output (overwritten by w)
  KrylovState* ks;             // 3 * ninst
  double* H;                   // 3 * ninst * (MAX_M+1) * MAX_M
  const int32_t* seg;          // 2 * ninst: [start, end) of each instance
  const int32_t* mask;         // ninst
  const double* h;             // ninst
  const int32_t* mstart;       // ninst: first dimension of the residual test (NULL = m_min)
  const int32_t *Gp, *Gi;
  const double* Gv;
  double eps;
  int m_min, m_max;
  unsigned* status;
  const int32_t* jdev;         // device iteration index (graph replays); NULL: use j
  unsigned long long* kv;      // count of directions built
  unsigned* where;             // first non-finite result: [flag, status bit, instance, slot * 256 + j]
  PadeCoef pade;
};

// record where the first non-finite value of a batched run appeared (first writer wins)
__device__ __forceinline__ void note_nonfinite(unsigned* where, unsigned bit, int inst, int slot,
                                               int j) {
  if (atomicCAS(where, 0u, 1u) == 0u) {
    where[1] = bit;
    where[2] = (unsigned)inst;
    where[3] = (unsigned)(slot * 256 + j);
  }
}

__device__ __forceinline__ double* bH_of(const BArgs& A, int slot, int i) {
  return A.H + ((int64_t)slot * A.ninst + i) * (MAX_M + 1) * MAX_M;
}

// ||G u||^2 over the rows of one segment
__device__ __forceinline__ double seg_gnorm2(const BArgs& A, const double* u, int s0, int s1) {
  double acc = 0.0;
  for (int i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
    double s = 0.0;
    for (int e = A.Gp[i]; e < A.Gp[i + 1]; ++e) s += A.Gv[e] * u[A.Gi[e]];
    acc += s * s;
  }
  return acc;
}

// beta = ||v_seg||, v_1 = v / beta, ||G v_1|| per (instance, space): one CTA each
__global__ void __launch_bounds__(BT) k_binit(BArgs A) {
  __shared__ double sh[BT / 32];
  const int i = blockIdx.x, b = blockIdx.y, slot = A.slot[b];
  KrylovState& K = A.ks[slot * A.ninst + i];
  const int s0 = A.seg[2 * i], s1 = A.seg[2 * i + 1];
  if (!A.mask[i]) {
    if (threadIdx.x == 0) { K.beta = 0.0; K.done = 1; K.m = 0; K.built = 0; K.breakdown = 0; }
    return;
  }
  const double* v = A.src[b];
  double* V0 = A.V[b];
  double acc = 0.0;
  for (int e = s0 + threadIdx.x; e < s1; e += blockDim.x) acc += v[e] * v[e];
  double beta = sqrt(block_sum(acc, sh));
  double inv = beta > 0.0 ? 1.0 / beta : 0.0;
  for (int e = s0 + threadIdx.x; e < s1; e += blockDim.x) V0[e] = v[e] * inv;
  double gv1 = 0.0;
  if (A.adaptive) {
    __syncthreads();
    gv1 = sqrt(block_sum(seg_gnorm2(A, V0, s0, s1), sh));
  }
  if (threadIdx.x == 0) {
    K.beta = beta;
    K.gv1 = gv1;
    K.built = 0;
    K.m = 0;
    K.best_m = 0;
    K.best_res = INFINITY;
    K.res = INFINITY;
    K.breakdown = 0;
    K.done = (beta > 0.0 && isfinite(beta)) ? 0 : 1;
    if (!isfinite(beta)) {
      atomicOr(A.status, ST_NONFINITE);
      note_nonfinite(A.where, ST_NONFINITE, i, slot, 0);
    }
  }
}

// modified Gram-Schmidt of w = -x (solve output) against v_1..v_{j+1} of one (instance, space)
__global__ void __launch_bounds__(BT) k_bmgs(BArgs A) {
  __shared__ double sh[BT / 32];
  const int i = blockIdx.x, b = blockIdx.y, slot = A.slot[b];
  KrylovState& K = A.ks[slot * A.ninst + i];
  if (!A.mask[i] || K.done) return;
  const int s0 = A.seg[2 * i], s1 = A.seg[2 * i + 1], n = A.n;
  const int j = A.jdev ? *A.jdev : A.j;
  double* w = A.src[b];
  const double* V = A.V[b];
  double* H = bH_of(A, slot, i);
  const int ldh = MAX_M + 1;
  double nn = 0.0, dd = 0.0;
  for (int e = s0 + threadIdx.x; e < s1; e += blockDim.x) {
    double x = -w[e];
    w[e] = x;
    nn += x * x;
    dd += x * V[e];
  }
  double w0 = sqrt(block_sum(nn, sh));
  double hcur = block_sum(dd, sh);
  if (threadIdx.x == 0) H[0 + j * ldh] = hcur;
  for (int it = 0; it <= j; ++it) {
    const double* vi = V + (int64_t)it * n;
    const double* vn = V + (int64_t)(it + 1) * n;
    double acc = 0.0;
    for (int e = s0 + threadIdx.x; e < s1; e += blockDim.x) {
      double x = w[e] - hcur * vi[e];
      w[e] = x;
      acc += (it < j) ? x * vn[e] : x * x;
    }
    hcur = block_sum(acc, sh);
    if (it < j && threadIdx.x == 0) H[(it + 1) + j * ldh] = hcur;
  }
  double hn = sqrt(hcur);
  bool bd = !(hn > 1e-12 * w0);
  double* vn = const_cast<double*>(V) + (int64_t)(j + 1) * n;
  if (!bd) {
    double inv = 1.0 / hn;
    for (int e = s0 + threadIdx.x; e < s1; e += blockDim.x) vn[e] = w[e] * inv;
  }
  double gn = 0.0;
  if (A.adaptive && !bd) {
    __syncthreads();
    gn = sqrt(block_sum(seg_gnorm2(A, vn, s0, s1), sh));
  }
  if (threadIdx.x == 0) {
    H[(j + 1) + j * ldh] = hn;
    K.w0 = w0;
    K.built = j + 1;
    K.gvnext[j] = gn;
    atomicAdd(A.kv, 1ull);
    if (!isfinite(hn)) {
      atomicOr(A.status, ST_NONFINITE);
      note_nonfinite(A.where, ST_NONFINITE, i, slot, j + 1);
    }
    if (bd) { K.breakdown = 1; K.done = 1; K.m = j + 1; }
  }
}

// Algorithm 1's dimension decision / exp(h_i H^-1) e_1 per (instance, space)
__global__ void k_bsmall(BArgs A) {
  extern __shared__ double smem[];
  __shared__ int ipiv[MAX_M];
  __shared__ double ybuf[MAX_M];
  __shared__ double s_last;
  const int i = blockIdx.x % A.ninst, b = blockIdx.x / A.ninst, slot = A.slot[b];
  if (!A.mask[i]) return;
  if (A.mode == SMALL_RESID && A.mstart) {
    // a proposed dimension: no residual test (Eq. 16) below it, unless the basis broke down
    const KrylovState& K = A.ks[slot * A.ninst + i];
    if (!K.done && !K.breakdown && K.built < min(A.mstart[i], A.m_max)) return;
  }
  KrylovState& K = A.ks[slot * A.ninst + i];
  small_decide(A.mode, bH_of(A, slot, i), K, A.h[i], A.eps, A.m_min, A.m_max,
               A.mstart ? A.mstart[i] : A.m_min, smem, ipiv, ybuf, &s_last, A.status, A.pade);
  __syncthreads();
  if (threadIdx.x == 0 && K.done && K.m > 0) {
    bool fin = isfinite(K.last);
    for (int k = 0; k < K.m; ++k) fin = fin && isfinite(K.y[k]);
    if (!fin) note_nonfinite(A.where, ST_KRYLOV, i, slot, K.built);
  }
}

// Parallel residual tests (Eq. 16) of the dimensions a proposed m_first skipped: one CTA per
// (instance, space, dimension d = d0 + blockIdx.z) of every space flagged by small_decide.
// Results go to per-(space, dimension) scratch: residual, finiteness, e_d^T H^-1 y and y.
struct ScanBuf {
  double* res;    // [slot][inst][MAX_M + 1]
  double* last;
  int32_t* fin;
  double* y;      // [slot][inst][MAX_M + 1][MAX_M]
};
__device__ __forceinline__ int64_t scan_idx(const BArgs& A, int slot, int i, int d) {
  return ((int64_t)slot * A.ninst + i) * (MAX_M + 1) + d;
}

__global__ void k_bscan(BArgs A, ScanBuf S, int d0) {
  extern __shared__ double smem[];
  __shared__ int ipiv[MAX_M];
  const int i = blockIdx.x, b = blockIdx.y, slot = A.slot[b], d = d0 + blockIdx.z;
  if (!A.mask[i]) return;
  const KrylovState& K = A.ks[slot * A.ninst + i];
  if (!K.scan || d > K.built || K.beta <= 0.0) return;
  const double* H = bH_of(A, slot, i);
  const int ldh = MAX_M + 1;
  const int64_t q = scan_idx(A, slot, i, d);
  bool fin = phi_small(H, ldh, d, A.h[i], S.y + q * MAX_M, S.last + q, smem, ipiv, A.pade);
  if (threadIdx.x == 0) {
    double res = H[d + (d - 1) * ldh] * K.gvnext[d - 1] * fabs(S.last[q]) / K.gv1;
    S.res[q] = fin ? res : INFINITY;
    S.fin[q] = fin ? 1 : 0;
  }
}

// The decision after a parallel scan: the first dimension in [m_min, built] that passes, as
// the plain rule's per-iteration tests would find it; at m_max with none passing, the
// never-converged choice of small_decide.  One warp per (instance, space).
__global__ void k_bpick(BArgs A, ScanBuf S) {
  const int i = blockIdx.x % A.ninst, b = blockIdx.x / A.ninst, slot = A.slot[b];
  const int lane = threadIdx.x;
  if (!A.mask[i]) return;
  KrylovState& K = A.ks[slot * A.ninst + i];
  if (!K.scan) return;
  const int built = K.built;
  int chosen = 0;
  double best = K.best_res;
  int best_m = K.best_m;
  for (int d = A.m_min; d <= built; ++d) {
    const int64_t q = scan_idx(A, slot, i, d);
    double r = S.res[q];
    if (isfinite(r) && r < best) { best = r; best_m = d; }
    if (isfinite(r) && r < A.eps) { chosen = d; break; }
  }
  bool finish = chosen > 0;
  if (!finish && built >= A.m_max) {
    chosen = best_m > 0 ? best_m : built;
    while (chosen > 1 && !S.fin[scan_idx(A, slot, i, chosen)]) --chosen;
    finish = true;
  }
  __syncwarp();
  if (finish) {
    const int64_t q = scan_idx(A, slot, i, chosen);
    for (int k = lane; k < chosen; k += 32) K.y[k] = S.y[q * MAX_M + k];
  }
  __syncwarp();
  if (lane == 0) {
    K.res = S.res[scan_idx(A, slot, i, chosen > 0 ? chosen : built)];
    K.best_res = best;
    K.best_m = best_m;
    if (finish) {
      const int64_t q = scan_idx(A, slot, i, chosen);
      K.last = S.last[q];
      K.m = chosen;
      K.done = 1;
      if (!S.fin[q]) {
        atomicOr(A.status, ST_KRYLOV);
        note_nonfinite(A.where, ST_KRYLOV, i, slot, chosen);
      }
    }
    K.scan = 0;
  }
}

__global__ void k_binc(int32_t* jdev) { *jdev += 1; }

// largest dimension chosen by the spaces of each instance
// (spaces 0 .. nb-1)
__global__ void k_bmused(int ninst, int nb, const KrylovState* ks, int32_t* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ninst) return;
  int m = 0;
  for (int b = 0; b < nb; ++b) m = max(m, ks[b * ninst + i].m);
  out[i] = m;
}

// how many (instance, space) pairs of the group are still iterating
// out[0] = spaces still running, out[1] = 1 when none is (the solves of later iterations
// that were already queued read it and do nothing)
__global__ void k_bcount(BArgs A, int32_t* out) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < A.ninst * A.nb; q += blockDim.x) {
    int i = q % A.ninst, b = q / A.ninst;
    if (A.mask[i] && !A.ks[A.slot[b] * A.ninst + i].done) atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = cnt;
    out[1] = cnt == 0;
  }
}

// out[e] = a in[e] + sum_b c_b beta_{b,i} V_b (y_{b,i} - e_1)[e] + hfac * h_i * u0[e]
// for the nodes e of instances i with mask[i] set (other nodes keep their value)
struct BCombine {
  int n, ninst, nb;
  double* out;
  const double* in;
  double a;
  const double* V[MAX_RHS];
  int slot[MAX_RHS];
  double c[MAX_RHS];
  const KrylovState* ks;
  const double* u0;
  double hfac;
  const double* h;
  const int32_t* inst_of;
  const int32_t* mask;
};

__global__ void __launch_bounds__(256) k_bcombine(BCombine A) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A.n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = A.inst_of[e];
    if (!A.mask[i]) continue;
    double v = A.in ? A.a * A.in[e] : 0.0;
    for (int b = 0; b < A.nb; ++b) {
      const KrylovState& K = A.ks[A.slot[b] * A.ninst + i];
      int m = K.beta > 0.0 ? K.m : 0;
      if (m == 0) continue;
      const double* Vb = A.V[b];
      double acc = (K.y[0] - 1.0) * Vb[e];
      for (int k = 1; k < m; ++k) acc += K.y[k] * Vb[(int64_t)k * A.n + e];
      v += A.c[b] * K.beta * acc;
    }
    if (A.u0) v += A.hfac * A.h[i] * A.u0[e];
    A.out[e] = v;
  }
}

// out[i] = max |x| over the nodes of instance i (0 when mask[i] is clear)
__global__ void __launch_bounds__(256) k_bmax(int ninst, const int32_t* seg, const int32_t* mask,
                                            const double* x, double* out) {
  __shared__ double sh[8];
  int i = blockIdx.x;
  double mx = 0.0;
  if (mask == nullptr || mask[i])
    for (int e = seg[2 * i] + threadIdx.x; e < seg[2 * i + 1]; e += blockDim.x) {
      double v = fabs(x[e]);
      mx = isfinite(v) ? fmax(mx, v) : INFINITY;
    }
  mx = block_max(mx, sh);
  if (threadIdx.x == 0) out[i] = mx;
}

__global__ void k_bcopy(int n, const int32_t* inst_of, const int32_t* mask, const double* src,
                        double* dst) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n && mask[inst_of[e]]) dst[e] = src[e];
}

// y_v = C (V_v)_j for the nv spaces; j from jdev when given (graph replays), else j
__global__ void k_brhs_C(int n, int nv, const int32_t* ptr, const int32_t* idx,
                         const double* val, const double* V0, const double* V1, const double* V2,
                         const int32_t* jdev, int j, double* y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t off = (int64_t)(jdev ? *jdev : j) * n;
  const double* xs[3] = {V0 + off, V1 ? V1 + off : nullptr, V2 ? V2 + off : nullptr};
  for (int v = 0; v < nv; ++v) {
    double acc = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) acc += val[e] * xs[v][idx[e]];
    y[(int64_t)v * n + i] = acc;
  }
}

__global__ void k_bbu(int n, const int32_t* ptr, const int32_t* idx, const double* val,
                      const double* u, const double* F, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = F ? F[i] : 0.0;
  for (int e = ptr[i]; e < ptr[i + 1]; ++e) acc += val[e] * u[idx[e]];
  out[i] = acc;
}

__global__ void k_bsub(int n, double* out, const double* x, const double* y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[i] - y[i];
}

}  // namespace ers

using namespace ers;

namespace {

inline int nblk(int n, int b = 256) { return std::max(1, (n + b - 1) / b); }

#define BCU(call)                                                                        \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return ctx_fail(c, e_ == cudaErrorMemoryAllocation ? ERS_ERR_OOM : ERS_ERR_CUDA,   \
                      std::string(#call) + ": " + cudaGetErrorString(e_));               \
  } while (0)

BArgs make_bargs(ers_ctx* c, int nb, const int* slots, double* const* src, int adaptive) {
  BArgs A{};
  A.n = c->n;
  A.ninst = c->ninst;
  A.nb = nb;
  A.adaptive = adaptive;
  for (int b = 0; b < nb; ++b) {
    A.slot[b] = slots[b];
    A.V[b] = c->V + (size_t)slots[b] * (MAX_M + 1) * c->n;
    A.src[b] = src ? src[b] : nullptr;
  }
  A.ks = c->bks;
  A.H = c->bH;
  A.seg = c->d_seg_off;
  A.mask = c->bmask;
  A.h = c->bh;
  A.Gp = c->G_ptr;
  A.Gi = c->G_idx;
  A.Gv = c->G_val;
  A.eps = c->opts.eps_krylov;
  A.m_min = c->opts.m_min;
  A.m_max = c->opts.m_max;
  A.status = c->d_status;
  A.pade = pade_coefficients(c->singular_c);
  A.mstart = c->ctrl ? c->d_mstart : nullptr;
  A.kv = c->d_kv;
  A.where = c->d_where;
  return A;
}

ers_status launch_bsmall(ers_ctx* c, BArgs A, int mode) {
  A.mode = mode;
  size_t sm = small_smem_doubles((size_t)c->opts.m_max) * 8;
  k_bsmall<<<c->ninst * A.nb, 256, sm, c->stream>>>(A);
  c->stats.kernel_launches++;
  BCU(cudaGetLastError());
  return ERS_OK;
}

ScanBuf scan_buf(ers_ctx* c) {
  return ScanBuf{c->bscan_res, c->bscan_last, c->bscan_fin, c->bscan_y};
}

// One Arnoldi iteration of the spaces of A: C v_j, the solves, Gram-Schmidt, the dimension
// test, and the count of spaces still running (c->bcount).  With use_jdev the iteration
// index is read from (and advanced in) device memory, which makes the sequence replayable as
// a graph.  The solve pass is skipped on the device once no space runs (c->bcount[1]).
cudaError_t enqueue_iteration(ers_ctx* c, const BArgs& A, int nb, int j, bool use_jdev) {
  const int32_t* jd = use_jdev ? c->bj : nullptr;
  k_brhs_C<<<nblk(c->n), 256, 0, c->stream>>>(c->n, nb, c->C_ptr, c->C_idx, c->C_val, A.V[0],
                                               nb > 1 ? A.V[1] : nullptr,
                                               nb > 2 ? A.V[2] : nullptr, jd, j, c->solve_buf);
  c->stats.kernel_launches++;
  const int* none_running[1] = {c->bcount + 1};
  cudaError_t e = launch_solve_skip(c, c->solve_buf, nb, none_running, 1);
  if (e != cudaSuccess) return e;
  BArgs M = A;
  M.j = j;
  M.jdev = jd;
  for (int b = 0; b < nb; ++b) M.src[b] = c->solve_buf + (size_t)b * c->n;
  k_bmgs<<<dim3(c->ninst, nb), BT, 0, c->stream>>>(M);
  c->stats.kernel_launches++;
  BArgs S = A;
  S.mode = SMALL_RESID;
  size_t mm = (size_t)c->opts.m_max;
  k_bsmall<<<c->ninst * nb, 256, small_smem_doubles(mm) * 8, c->stream>>>(S);
  c->stats.kernel_launches++;
  k_bcount<<<1, 256, 0, c->stream>>>(A, c->bcount);
  c->stats.kernel_launches++;
  if (use_jdev) {
    k_binc<<<1, 1, 0, c->stream>>>(c->bj);
    c->stats.kernel_launches++;
  }
  return cudaGetLastError();
}

// The graph of one iteration for this combination of spaces (captured on first use).  Returns
// nullptr when graphs are off or the capture fails (then graphs stay off for the context).
ers_ctx::IterGraph* iteration_graph(ers_ctx* c, const BArgs& A, int nb, const int* slots) {
  if (!c->batch_graphs) return nullptr;
  const int ctrl = c->ctrl != nullptr;
  for (auto& g : c->iter_graphs) {
    bool same = g.nb == nb && g.ctrl == ctrl;
    for (int b = 0; b < nb && same; ++b) same = g.slot[b] == slots[b];
    if (same) return &g;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (c->stream == nullptr || cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    c->batch_graphs = false;     // legacy default stream, or a capture of the caller's
    cudaGetLastError();
    return nullptr;
  }
  const ers_stats_t s0 = c->stats;
  const bool prof = c->profile;
  c->profile = false;   // no event records inside the graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t ee = enqueue_iteration(c, A, nb, 0, true);
    e = cudaStreamEndCapture(c->stream, &graph);
    if (e == cudaSuccess) e = ee;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  c->profile = prof;
  ers_ctx::IterGraph g;
  g.launches = c->stats.kernel_launches - s0.kernel_launches;
  g.solves = c->stats.solves - s0.solves;
  g.passes = c->stats.solve_passes - s0.solve_passes;
  g.rhs = c->stats.solve_rhs - s0.solve_rhs;
  c->stats = s0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    c->batch_graphs = false;
    return nullptr;
  }
  g.nb = nb;
  g.ctrl = ctrl;
  for (int b = 0; b < nb; ++b) g.slot[b] = slots[b];
  g.exec = exec;
  c->iter_graphs.push_back(g);
  return &c->iter_graphs.back();
}

// Algorithm 1 up to the MEVP for the spaces `slots` of every instance set in `mask` (the host
// copy of the device mask; adaptive m).  No space can finish before its first decision (at
// m_min, or at the proposed dimension) unless it breaks down, and a broken-down space only
// skips work, so the host polls for completion from the smallest first decision on.  The
// poll is lagged: every iteration ends with an asynchronous copy of the running count into a
// pinned ring slot and an event, and before iteration j the host reads iteration
// j - BPOLL_LAG's count, so the device always has the next iteration queued; the kernels of a
// finished space, and the solve pass once none runs, do nothing.
constexpr int BPOLL_LAG = 2, BPOLL_RING = 4;

ers_status batch_bases(ers_ctx* c, int nb, const int* slots, double* const* src,
                       const std::vector<int32_t>& mask) {
  const int mc = c->opts.m_max;
  int first_test = mc;
  for (int i = 0; i < c->ninst; ++i)
    if (mask[i])
      first_test = std::min(first_test, c->ctrl ? std::max(c->mstart_inst[i], c->opts.m_min)
                                                : c->opts.m_min);
  c->scan_mask = mask;
  BArgs A = make_bargs(c, nb, slots, src, 1);
  k_binit<<<dim3(c->ninst, nb), BT, 0, c->stream>>>(A);
  c->stats.kernel_launches++;
  ers_ctx::IterGraph* G = iteration_graph(c, A, nb, slots);
  if (G) BCU(cudaMemsetAsync(c->bj, 0, sizeof(int32_t), c->stream));
  BCU(cudaMemsetAsync(c->bcount, 0, 2 * sizeof(int32_t), c->stream));
  for (int s = 0; s < BPOLL_RING; ++s)
    if (!c->poll_ev[s]) BCU(cudaEventCreateWithFlags(&c->poll_ev[s], cudaEventDisableTiming));
  int32_t* ring = reinterpret_cast<int32_t*>(c->h_scalars + 32);   // BPOLL_RING counts
  for (int j = 0; j < mc; ++j) {
    // the count after iteration j - BPOLL_LAG reflects the tests up to dimension
    // j - BPOLL_LAG + 1; the first space can finish at dimension first_test
    if (j >= BPOLL_LAG && j - BPOLL_LAG + 1 >= first_test) {
      const int slot = (j - BPOLL_LAG) % BPOLL_RING;
      BCU(cudaEventSynchronize(c->poll_ev[slot]));
      c->stats.host_polls++;
      if (ring[slot] == 0) break;
    }
    if (G) {
      BCU(cudaGraphLaunch(G->exec, c->stream));
      c->stats.graph_launches++;
      c->stats.kernel_launches += G->launches;
      c->stats.solves += G->solves;
      c->stats.solve_passes += G->passes;
      c->stats.solve_rhs += G->rhs;
    } else {
      BCU(enqueue_iteration(c, A, nb, j, false));
    }
    {
      const int slot = j % BPOLL_RING;
      BCU(cudaMemcpyAsync(ring + slot, c->bcount, sizeof(int32_t), cudaMemcpyDeviceToHost,
                          c->stream));
      BCU(cudaEventRecord(c->poll_ev[slot], c->stream));
    }
    // instances whose proposed first decision is at dimension j + 1: test [m_min, j + 1]
    if (c->ctrl && j + 1 > c->opts.m_min) {
      bool any = false;
      for (int i = 0; i < c->ninst && !any; ++i)
        any = c->scan_mask[i] && c->mstart_inst[i] == j + 1;
      if (any) {
        const int nd = j + 1 - c->opts.m_min + 1;
        size_t mm = (size_t)c->opts.m_max;
        size_t sm = small_smem_doubles(mm) * 8;
        k_bscan<<<dim3(c->ninst, nb, nd), 256, sm, c->stream>>>(A, scan_buf(c), c->opts.m_min);
        k_bpick<<<c->ninst * nb, 32, 0, c->stream>>>(A, scan_buf(c));
        c->stats.kernel_launches += 2;
        BCU(cudaGetLastError());
      }
    }
  }
  return ERS_OK;
}

// a failed status of a batched run, with the first non-finite location added to the message
ers_status batch_fail_where(ers_ctx* c, ers_status st) {
  unsigned w[4] = {0, 0, 0, 0};
  if (cudaMemcpy(w, c->d_where, sizeof(w), cudaMemcpyDeviceToHost) == cudaSuccess && w[0]) {
    const char* what = w[1] == ST_KRYLOV ? "exp(h H^-1) e_1" : "Krylov vector";
    c->err += std::string(" (first non-finite ") + what + ": instance " + std::to_string(w[2]) +
              ", space " + std::to_string(w[3] / 256) + ", dimension " +
              std::to_string(w[3] % 256) + ")";
  }
  return st;
}

double next_bp(const std::vector<double>& bp, double t) {
  auto it = std::upper_bound(bp.begin(), bp.end(), t * (1 + 1e-14) + 1e-30);
  return it == bp.end() ? INFINITY : *it;
}

}  // namespace

// A batched context of ninst instances on the current device.
ers_status ers::create_batch_here(ers_ctx** out, const ers_instance* inst, int32_t ninst,
                                  const ers_opts* opts) {
  if (!out) return ERS_ERR_INVALID;
  ers_ctx* c = new ers_ctx();
  *out = c;
  if (!inst || ninst < 1) return ctx_fail(c, ERS_ERR_INVALID, "need at least one instance");
  if (opts && (opts->correction || opts->combined_vector))
    return ctx_fail(c, ERS_ERR_INVALID,
                    "batched runs use the ER step with separate phi_1 / phi_2 spaces "
                    "(correction and combined_vector are single-context options)");
  // concatenate the instances into one block-diagonal circuit
  std::vector<int32_t> gp{0}, gi, cp{0}, ci, bp{0}, bi;
  std::vector<double> gv, cv, bv;
  std::vector<ers_mosfet> devs;
  std::vector<ers_pwl> pw;
  std::vector<int32_t> orig{0}, src_inst;
  int ntot = 0, ptot = 0;
  for (int k = 0; k < ninst; ++k) {
    const ers_instance& I = inst[k];
    if (!I.G || !I.C || !I.B || I.G->n_rows <= 0 || I.C->n_rows != I.G->n_rows ||
        I.B->n_rows != I.G->n_rows || I.p < 0 || I.B->n_cols != I.p || (I.p > 0 && !I.u) ||
        I.ndev < 0 || (I.ndev > 0 && !I.dev))
      return ctx_fail(c, ERS_ERR_INVALID, "instance " + std::to_string(k) + " is malformed");
    int n = I.G->n_rows;
    auto append = [&](const ers_csr* A, int col_off, std::vector<int32_t>& P,
                      std::vector<int32_t>& X, std::vector<double>& Vv) {
      for (int r = 0; r < A->n_rows; ++r) {
        for (int e = A->rowptr[r]; e < A->rowptr[r + 1]; ++e) {
          X.push_back(A->colidx[e] + col_off);
          Vv.push_back(A->val[e]);
        }
        P.push_back((int32_t)X.size());
      }
    };
    append(I.G, ntot, gp, gi, gv);
    append(I.C, ntot, cp, ci, cv);
    append(I.B, ptot, bp, bi, bv);
    for (int d = 0; d < I.ndev; ++d) {
      ers_mosfet m = I.dev[d];
      if (m.d >= 0) m.d += ntot;
      if (m.g >= 0) m.g += ntot;
      if (m.s >= 0) m.s += ntot;
      devs.push_back(m);
    }
    for (int q = 0; q < I.p; ++q) {
      pw.push_back(I.u[q]);
      src_inst.push_back(k);
    }
    ntot += n;
    ptot += I.p;
    orig.push_back(ntot);
  }
  ers_csr G{ntot, ntot, (int32_t)gi.size(), gp.data(), gi.data(), gv.data()};
  ers_csr C{ntot, ntot, (int32_t)ci.size(), cp.data(), ci.data(), cv.data()};
  ers_csr B{ntot, ptot, (int32_t)bi.size(), bp.data(), bi.data(), bv.data()};
  ers_status st = create_context(c, &G, &C, &B, devs.empty() ? nullptr : devs.data(),
                                 (int32_t)devs.size(), pw.empty() ? nullptr : pw.data(), ptot,
                                 opts);
  if (st != ERS_OK) return st;
  // every instance must occupy one contiguous range of the internal order
  const Symbolic& S = c->sym;
  c->ninst = ninst;
  c->orig_off = orig;
  c->seg_off.assign(ninst + 1, 0);
  std::vector<int32_t> inst_of(ntot);
  for (int k = 0; k < ninst; ++k) {
    int lo = ntot, hi = -1;
    for (int v = orig[k]; v < orig[k + 1]; ++v) {
      lo = std::min(lo, S.iperm[v]);
      hi = std::max(hi, S.iperm[v]);
    }
    if (hi - lo + 1 != orig[k + 1] - orig[k])
      return ctx_fail(c, ERS_ERR_INVALID, "internal: instance nodes are not contiguous");
    for (int q = lo; q <= hi; ++q) inst_of[q] = k;
    c->seg_off[k] = lo;
  }
  // device segment table in instance order: [start_k, start_k + n_k)
  std::vector<int32_t> seg_lo(ninst), seg_hi(ninst);
  for (int k = 0; k < ninst; ++k) {
    seg_lo[k] = c->seg_off[k];
    seg_hi[k] = c->seg_off[k] + (orig[k + 1] - orig[k]);
  }
  // kernels take seg[i], seg[i+1]: store as pairs (2 ninst ints) via an interleaved table
  std::vector<int32_t> segtab(2 * ninst);
  for (int k = 0; k < ninst; ++k) { segtab[2 * k] = seg_lo[k]; segtab[2 * k + 1] = seg_hi[k]; }
  c->bp_inst.assign(ninst, {});
  for (int q = 0; q < ptot; ++q) {
    int k = src_inst[q];
    for (int a = 0; a < pw[q].npts; ++a) c->bp_inst[k].push_back(pw[q].t[a]);
  }
  for (auto& v : c->bp_inst) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  c->t_inst.assign(ninst, 0.0);
  c->hprop_inst.assign(ninst, 0.0);
  c->steps_inst.assign(ninst, 0);
  c->rejects_inst.assign(ninst, 0);
  auto up = [&](auto** dst, const auto& v) -> cudaError_t {
    using T = typename std::decay<decltype(v[0])>::type;
    cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(1, v.size()) * sizeof(T));
    if (e == cudaSuccess && !v.empty())
      e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
  };
  BCU(up(&c->d_inst_of, inst_of));
  BCU(up(&c->d_seg_off, segtab));
  BCU(up(&c->d_src_inst, src_inst));
  BCU(cudaMalloc((void**)&c->bks, sizeof(KrylovState) * 3 * (size_t)ninst));
  BCU(cudaMemset(c->bks, 0, sizeof(KrylovState) * 3 * (size_t)ninst));
  BCU(cudaMalloc((void**)&c->bH, sizeof(double) * 3 * (size_t)ninst * (MAX_M + 1) * MAX_M));
  BCU(cudaMemset(c->bH, 0, sizeof(double) * 3 * (size_t)ninst * (MAX_M + 1) * MAX_M));
  BCU(cudaMalloc((void**)&c->bh, sizeof(double) * ninst));
  BCU(cudaMalloc((void**)&c->bt, sizeof(double) * ninst));
  BCU(cudaMalloc((void**)&c->bred, sizeof(double) * ninst));
  BCU(cudaMalloc((void**)&c->bmask, sizeof(int32_t) * ninst));
  BCU(cudaMalloc((void**)&c->bcount, 2 * sizeof(int32_t)));
  BCU(cudaMallocHost((void**)&c->h_bpin, sizeof(double) * 4 * (size_t)ninst));
  c->h_src_inst = src_inst;
  BCU(cudaMalloc((void**)&c->d_mstart, sizeof(int32_t) * ninst));
  BCU(cudaMalloc((void**)&c->d_kv, sizeof(unsigned long long)));
  BCU(cudaMalloc((void**)&c->bj, sizeof(int32_t)));
  BCU(cudaMalloc((void**)&c->d_where, 4 * sizeof(unsigned)));
  BCU(cudaMemset(c->d_where, 0, 4 * sizeof(unsigned)));
  BCU(cudaMemset(c->d_kv, 0, sizeof(unsigned long long)));
  BCU(cudaMalloc((void**)&c->d_mused, sizeof(int32_t) * ninst));
  BCU(cudaMalloc((void**)&c->bdf, sizeof(double) * ninst));
  BCU(cudaMalloc((void**)&c->d_feat, sizeof(float) * ERS_CTRL_FEATURES * (size_t)ninst));
  BCU(cudaMalloc((void**)&c->d_pred, sizeof(float) * 2 * (size_t)ninst));
  c->recs.assign(ninst, {});
  c->mstart_inst.assign(ninst, c->opts.m_min);
  c->proposed_inst.assign(ninst, 0);
  BCU(cudaFuncSetAttribute(k_bsmall, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           small_smem_doubles(MAX_M) * 8));
  BCU(cudaFuncSetAttribute(k_bscan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           small_smem_doubles(MAX_M) * 8));
  {
    const size_t nq = (size_t)3 * ninst * (MAX_M + 1);
    BCU(cudaMalloc((void**)&c->bscan_res, sizeof(double) * nq));
    BCU(cudaMalloc((void**)&c->bscan_last, sizeof(double) * nq));
    BCU(cudaMalloc((void**)&c->bscan_fin, sizeof(int32_t) * nq));
    BCU(cudaMalloc((void**)&c->bscan_y, sizeof(double) * nq * MAX_M));
  }
  return ERS_OK;
}

extern "C" {

ers_status ers_create_batch(ers_ctx** out, const ers_instance* inst, int32_t ninst,
                            const int32_t* devices, int32_t ndevices, const ers_opts* opts) {
  if (!out) return ERS_ERR_INVALID;
  *out = nullptr;
  std::string bad = check_device_list(devices, ndevices);
  if (!bad.empty()) {
    ers_ctx* c = new ers_ctx();
    *out = c;
    return ctx_fail(c, ERS_ERR_INVALID, bad);
  }
  if (ndevices > 1 && inst && ninst >= 1) {
    ers_ctx* g = new ers_ctx();
    *out = g;
    return group_create(g, inst, ninst, devices, ndevices, opts);
  }
  DeviceGuard dg(ndevices == 1 ? devices[0] : -1);
  return create_batch_here(out, inst, ninst, opts);
}

ers_status ers_run_batch(ers_ctx* c, double t_end, double tol, int32_t max_steps,
                         int32_t* nsteps, int32_t* nreject) {
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group()) return group_run_batch(c, t_end, tol, max_steps, nsteps, nreject);
  DeviceGuard dg(c->device);
  if (!c->bks) return ctx_fail(c, ERS_ERR_INVALID, "context was not created by ers_create_batch");
  if (!(tol > 0.0)) return ctx_fail(c, ERS_ERR_INVALID, "tol must be positive");
  const int ninst = c->ninst, n = c->n;
  const ers_opts& o = c->opts;
  const double h_max = o.h_max > 0 ? o.h_max : t_end / 100.0;
  std::vector<double> h(ninst), E(ninst), err(ninst), dF(ninst), dF_acc(ninst);
  std::vector<double> err_acc(ninst);
  std::vector<int32_t> active(ninst), trying(ninst), retries(ninst), mused(ninst);
  std::vector<int> landed(ninst);
  std::vector<float> feat, pred;
  ers_status st = ctx_clear_status(c);
  if (st != ERS_OK) return st;
  BCU(cudaMemsetAsync(c->d_where, 0, 4 * sizeof(unsigned), c->stream));
  const std::vector<int64_t> steps0 = c->steps_inst, rejects0 = c->rejects_inst;
  // pinned per-instance words filled by asynchronous copies and read after a try's sync
  double* pin_xmax = c->h_bpin;
  double* pin_dF = c->h_bpin + ninst;
  double* pin_err = c->h_bpin + 2 * (size_t)ninst;
  int32_t* pin_mused = reinterpret_cast<int32_t*>(c->h_bpin + 3 * (size_t)ninst);
  int round = 0;
  std::vector<int32_t> ones(ninst, 1);
  while (max_steps <= 0 || round < max_steps) {
    int nact = 0;
    for (int i = 0; i < ninst; ++i) {
      active[i] = c->t_inst[i] < t_end * (1 - 1e-12);
      nact += active[i];
      if (!active[i]) { h[i] = 0.0; continue; }
      double nb = std::min(next_bp(c->bp_inst[i], c->t_inst[i]), t_end);
      double hp = c->hprop_inst[i] > 0 ? c->hprop_inst[i] : (o.h_init > 0 ? o.h_init : h_max);
      h[i] = std::min(std::min(hp, h_max), nb - c->t_inst[i]);
      landed[i] = h[i] == nb - c->t_inst[i];
      retries[i] = 0;
      if (!c->ctrl) c->mstart_inst[i] = o.m_min;
    }
    if (nact == 0) break;
    // error budgets from ||x_i||_inf, read with the first try's synchronisation (pinned);
    // the uploads below are stream-ordered and need no synchronisation
    BCU(cudaMemcpyAsync(c->bmask, ones.data(), sizeof(int32_t) * ninst, cudaMemcpyHostToDevice, c->stream));
    k_bmax<<<ninst, 256, 0, c->stream>>>(ninst, c->d_seg_off, c->bmask, c->x, c->bred);
    BCU(cudaMemcpyAsync(pin_xmax, c->bred, sizeof(double) * ninst, cudaMemcpyDeviceToHost, c->stream));
    BCU(cudaMemcpyAsync(c->bh, h.data(), sizeof(double) * ninst, cudaMemcpyHostToDevice, c->stream));
    BCU(cudaMemcpyAsync(c->bt, c->t_inst.data(), sizeof(double) * ninst, cudaMemcpyHostToDevice, c->stream));
    BCU(cudaMemcpyAsync(c->bmask, active.data(), sizeof(int32_t) * ninst, cudaMemcpyHostToDevice, c->stream));
    if (c->ctrl)
      BCU(cudaMemcpyAsync(c->d_mstart, c->mstart_inst.data(), sizeof(int32_t) * ninst,
                          cudaMemcpyHostToDevice, c->stream));
    bool have_E = false;
    if (!c->factored) {
      st = ctx_refactor(c);
      if (st != ERS_OK) return st;
    }
    // setup vectors (Eq. 12-13): v1 = x - G^-1 (F + B u), w1 = G^-1 B s, v2 = G^-1 C w1
    k_bpwl<<<nblk(c->p), 256, 0, c->stream>>>(c->p, c->pwl_ptr, c->pwl_t, c->pwl_v, c->d_src_inst,
                                              c->bt, c->bh, c->bmask, c->u, c->slope);
    k_bbu<<<nblk(n), 256, 0, c->stream>>>(n, c->B_ptr, c->B_idx, c->B_val, c->u, c->F, c->solve_buf);
    k_bbu<<<nblk(n), 256, 0, c->stream>>>(n, c->B_ptr, c->B_idx, c->B_val, c->slope, nullptr,
                                          c->solve_buf + n);
    // whether some active instance's source has a non-zero slope: decided on the host with
    // the kernel's own arithmetic (pwl_eval at t_i and t_i + h_i), no read-back
    bool ramp = false;
    for (int q = 0; q < c->p && !ramp; ++q) {
      const int i = c->h_src_inst[q];
      if (!active[i] || !(h[i] > 0.0)) continue;
      const int o = c->h_pwl_ptr[q], np = c->h_pwl_ptr[q + 1] - o;
      const double* tt = c->h_pwl_t.data() + o;
      const double* vv = c->h_pwl_v.data() + o;
      ramp = pwl_eval(tt, vv, np, c->t_inst[i] + h[i]) != pwl_eval(tt, vv, np, c->t_inst[i]);
    }
    BCU(launch_solve(c, c->solve_buf, ramp ? 2 : 1));
    k_bsub<<<nblk(n), 256, 0, c->stream>>>(n, c->v1, c->x, c->solve_buf);
    if (ramp) {
      BCU(cudaMemcpyAsync(c->w1, c->solve_buf + n, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
      launch_spmv(c, c->C_ptr, c->C_idx, c->C_val, c->w1, c->solve_buf, 1.0);
      BCU(launch_solve(c, c->solve_buf, 1));
      BCU(cudaMemcpyAsync(c->v2, c->solve_buf, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    c->stats.kernel_launches += 5;
    int slots[2] = {0, 1};
    double* src[2] = {c->v1, c->v2};
    const int nsol = ramp ? 2 : 1;
    st = batch_bases(c, nsol, slots, src, active);
    if (st != ERS_OK) return st;
    k_bmused<<<nblk(ninst), 256, 0, c->stream>>>(ninst, nsol, c->bks, c->d_mused);
    BCU(cudaMemcpyAsync(pin_mused, c->d_mused, sizeof(int32_t) * ninst, cudaMemcpyDeviceToHost, c->stream));
    c->stats.kernel_launches++;
    trying = active;
    while (true) {
      BCU(cudaMemcpyAsync(c->bmask, trying.data(), sizeof(int32_t) * ninst, cudaMemcpyHostToDevice, c->stream));
      BCU(cudaMemcpyAsync(c->bh, h.data(), sizeof(double) * ninst, cudaMemcpyHostToDevice, c->stream));
      BCombine U{};
      U.n = n; U.ninst = ninst; U.nb = nsol; U.out = c->xnew; U.in = c->x; U.a = 1.0;
      for (int b = 0; b < nsol; ++b) {
        U.V[b] = c->V + (size_t)slots[b] * (MAX_M + 1) * n;
        U.slot[b] = slots[b];
        U.c[b] = 1.0;
      }
      U.ks = c->bks; U.u0 = ramp ? c->w1 : nullptr; U.hfac = 1.0; U.h = c->bh;
      U.inst_of = c->d_inst_of; U.mask = c->bmask;
      k_bcombine<<<std::min(c->sm_count * 8, nblk(n)), 256, 0, c->stream>>>(U);
      c->stats.kernel_launches++;
      std::fill(pin_err, pin_err + ninst, 0.0);
      std::fill(pin_dF, pin_dF + ninst, 0.0);
      if (c->ndev) {
        // e_rr = -(e^{hJ} - I) G^-1 dF per instance (Eq. 15)
        launch_dev_eval(c, c->xnew, c->dev_I + c->ndev, 0);
        launch_node_F(c, 1, c->dev_I + c->ndev, c->xnew, c->solve_buf);
        k_bmax<<<ninst, 256, 0, c->stream>>>(ninst, c->d_seg_off, c->bmask, c->solve_buf, c->bdf);
        BCU(cudaMemcpyAsync(pin_dF, c->bdf, sizeof(double) * ninst, cudaMemcpyDeviceToHost, c->stream));
        BCU(launch_solve(c, c->solve_buf, 1));
        BCU(cudaMemcpyAsync(c->ve, c->solve_buf, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        int es = 2;
        double* esrc[1] = {c->ve};
        st = batch_bases(c, 1, &es, esrc, trying);
        if (st != ERS_OK) return st;
        BCombine Er{};
        Er.n = n; Er.ninst = ninst; Er.nb = 1; Er.out = c->tmp; Er.in = nullptr; Er.a = 0.0;
        Er.V[0] = c->V + (size_t)2 * (MAX_M + 1) * n; Er.slot[0] = 2; Er.c[0] = -1.0;
        Er.ks = c->bks; Er.u0 = nullptr; Er.h = c->bh; Er.inst_of = c->d_inst_of; Er.mask = c->bmask;
        k_bcombine<<<std::min(c->sm_count * 8, nblk(n)), 256, 0, c->stream>>>(Er);
        k_bmax<<<ninst, 256, 0, c->stream>>>(ninst, c->d_seg_off, c->bmask, c->tmp, c->bred);
        BCU(cudaMemcpyAsync(pin_err, c->bred, sizeof(double) * ninst, cudaMemcpyDeviceToHost, c->stream));
        c->stats.kernel_launches += 3;
      }
      st = ctx_sync_status(c);    // the try's one synchronisation
      if (st != ERS_OK) return batch_fail_where(c, st);
      std::copy(pin_err, pin_err + ninst, err.begin());
      std::copy(pin_dF, pin_dF + ninst, dF.begin());
      if (!have_E) {
        for (int i = 0; i < ninst; ++i)
          E[i] = o.E_rr > 0 ? o.E_rr : tol * std::max(1.0, pin_xmax[i]);
        std::copy(pin_mused, pin_mused + ninst, mused.begin());
        have_E = true;
      }
      int left = 0;
      for (int i = 0; i < ninst; ++i) {
        if (!trying[i]) continue;
        if (err[i] <= E[i]) {
          trying[i] = 0;
          err_acc[i] = err[i];
          dF_acc[i] = dF[i];
          continue;
        }
        if (retries[i] == 0 && c->proposed_inst[i]) c->ctrl_rejected++;
        h[i] *= o.alpha;
        retries[i]++;
        c->rejects_inst[i]++;
        landed[i] = 0;
        if (h[i] < o.h_min) return ctx_fail(c, ERS_ERR_STEP_UNDERFLOW, "step size underflow in instance " + std::to_string(i));
        left++;
      }
      if (!left) break;
      // rejected instances: same bases and m, exp(h H^-1) at the new h (Alg. 2)
      BCU(cudaMemcpyAsync(c->bmask, trying.data(), sizeof(int32_t) * ninst, cudaMemcpyHostToDevice, c->stream));
      BCU(cudaMemcpyAsync(c->bh, h.data(), sizeof(double) * ninst, cudaMemcpyHostToDevice, c->stream));
      BArgs R = make_bargs(c, nsol, slots, nullptr, 1);
      st = launch_bsmall(c, R, SMALL_FINAL);
      if (st != ERS_OK) return st;
    }
    BCU(cudaMemcpyAsync(c->bmask, active.data(), sizeof(int32_t) * ninst, cudaMemcpyHostToDevice, c->stream));
    k_bcopy<<<nblk(n), 256, 0, c->stream>>>(n, c->d_inst_of, c->bmask, c->xnew, c->x);
    c->stats.kernel_launches++;
    std::vector<int> ask;
    for (int i = 0; i < ninst; ++i) {
      if (!active[i]) continue;
      double nb = std::min(next_bp(c->bp_inst[i], c->t_inst[i]), t_end);
      c->t_inst[i] = landed[i] ? nb : c->t_inst[i] + h[i];
      c->steps_inst[i]++;
      // plain controller of Alg. 2
      c->hprop_inst[i] = retries[i] < o.i_grow ? std::min(o.beta * h[i], h_max) : h[i];
      c->proposed_inst[i] = 0;
      ers_step_record r{};
      r.h = h[i];
      r.h_max = h_max;
      r.err = err_acc[i];
      r.E = E[i];
      r.dF = dF_acc[i];
      r.m = mused[i];
      r.m_max = o.m_max;
      r.landed = landed[i];
      r.retries = retries[i];
      auto& R = c->recs[i];
      R.push_back(r);
      if (!c->trace && R.size() > 2 * ERS_CTRL_HISTORY)
        R.erase(R.begin(), R.end() - ERS_CTRL_HISTORY);
      if (c->ctrl && c->t_inst[i] < t_end * (1 - 1e-12)) ask.push_back(i);
    }
    if (!ask.empty()) {
      // learned controller: the network proposes (h, m) of the next step of each instance
      const int na = (int)ask.size();
      feat.resize((size_t)na * ERS_CTRL_FEATURES);
      pred.resize((size_t)na * 2);
      for (int q = 0; q < na; ++q) {
        const auto& R = c->recs[ask[q]];
        ctrl_features(R.data(), (int)R.size(), &feat[(size_t)q * ERS_CTRL_FEATURES]);
      }
      BCU(cudaMemcpyAsync(c->d_feat, feat.data(), sizeof(float) * feat.size(), cudaMemcpyHostToDevice, c->stream));
      st = ers_mlp_forward_dev(c->ctrl, c->d_feat, na, c->d_pred, c->stream);
      if (st != ERS_OK) return ctx_fail(c, st, std::string("controller network: ") + ers_mlp_last_error(c->ctrl));
      BCU(cudaMemcpyAsync(pred.data(), c->d_pred, sizeof(float) * pred.size(), cudaMemcpyDeviceToHost, c->stream));
      BCU(cudaStreamSynchronize(c->stream));
      c->stats.host_syncs++;
      c->stats.kernel_launches++;
      for (int q = 0; q < na; ++q) {
        int i = ask[q];
        double hn;
        int ms;
        const ers_step_record& last = c->recs[i].back();
        ctrl_propose(&pred[2 * q], h[i], h_max, o.m_min, o.m_max, c->ctrl_margin,
                     last.E > 0.0 ? last.err / last.E : 0.0, &hn, &ms);
        if (c->ctrl_parts & ERS_CTRL_H) {
          c->hprop_inst[i] = hn;
          c->proposed_inst[i] = 1;
          c->ctrl_proposals++;
        }
        c->mstart_inst[i] = (c->ctrl_parts & ERS_CTRL_M) ? ms : o.m_min;
      }
    }
    if (!c->linear) c->factored = false;
    c->stats.steps++;
    ++round;
  }
  unsigned long long kv = 0;
  BCU(cudaMemcpyAsync(&kv, c->d_kv, sizeof(kv), cudaMemcpyDeviceToHost, c->stream));
  BCU(cudaStreamSynchronize(c->stream));
  c->stats.krylov_vectors = (int64_t)kv;
  for (int i = 0; i < ninst; ++i) {
    if (nsteps) nsteps[i] = (int32_t)(c->steps_inst[i] - steps0[i]);
    if (nreject) nreject[i] = (int32_t)(c->rejects_inst[i] - rejects0[i]);
    c->stats.rejects += c->rejects_inst[i] - rejects0[i];
  }
  return ERS_OK;
}

ers_status ers_batch_set_controller(ers_ctx* c, ers_mlp* mlp, int32_t parts, double margin) {
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group()) return group_set_controller(c, mlp, parts, margin);
  if (!c->bks) return ctx_fail(c, ERS_ERR_INVALID, "context was not created by ers_create_batch");
  if (mlp && (parts & ~(ERS_CTRL_H | ERS_CTRL_M)) != 0)
    return ctx_fail(c, ERS_ERR_INVALID, "unknown controller parts");
  if (!(margin >= 0.0) || !std::isfinite(margin))
    return ctx_fail(c, ERS_ERR_INVALID, "margin must be finite and >= 0");
  c->ctrl_margin = margin;
  c->ctrl = (parts & (ERS_CTRL_H | ERS_CTRL_M)) ? mlp : nullptr;
  c->ctrl_parts = parts;
  std::fill(c->proposed_inst.begin(), c->proposed_inst.end(), 0);
  std::fill(c->mstart_inst.begin(), c->mstart_inst.end(), c->opts.m_min);
  return ERS_OK;
}

ers_status ers_batch_set_graphs(ers_ctx* c, int32_t enable) {
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group())
    return group_call(c, [&](ers_ctx* s, int) { return ers_batch_set_graphs(s, enable); });
  if (!c->bks) return ctx_fail(c, ERS_ERR_INVALID, "context was not created by ers_create_batch");
  c->batch_graphs = enable != 0;
  return ERS_OK;
}

ers_status ers_batch_trace(ers_ctx* c, int32_t enable) {
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group())
    return group_call(c, [&](ers_ctx* s, int) { return ers_batch_trace(s, enable); });
  if (!c->bks) return ctx_fail(c, ERS_ERR_INVALID, "context was not created by ers_create_batch");
  c->trace = enable != 0;
  for (auto& R : c->recs) R.clear();
  return ERS_OK;
}

ers_status ers_batch_records(const ers_ctx* cc, int32_t k, ers_step_record* out, int32_t cap,
                             int32_t* count) {
  ers_ctx* c = const_cast<ers_ctx*>(cc);
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group()) return group_records(c, k, out, cap, count);
  if (!c->bks) return ctx_fail(c, ERS_ERR_INVALID, "context was not created by ers_create_batch");
  if (k < 0 || k >= c->ninst) return ctx_fail(c, ERS_ERR_INVALID, "instance index out of range");
  const auto& R = c->recs[k];
  if (count) *count = (int32_t)R.size();
  if (out)
    for (int32_t q = 0; q < std::min<int32_t>(cap, (int32_t)R.size()); ++q) out[q] = R[q];
  return ERS_OK;
}

ers_status ers_batch_samples(const ers_ctx* cc, float* X, float* T, int32_t cap, int32_t* count) {
  ers_ctx* c = const_cast<ers_ctx*>(cc);
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group()) return group_samples(c, X, T, cap, count);
  if (!c->bks) return ctx_fail(c, ERS_ERR_INVALID, "context was not created by ers_create_batch");
  int64_t ns = 0;
  for (const auto& R : c->recs) {
    for (size_t k = 0; k + 1 < R.size(); ++k) {
      float t[2];
      if (!ctrl_target(R.data(), (int)k + 1, R[k + 1], t)) continue;
      if (X && T && ns < cap) {
        ctrl_features(R.data(), (int)k + 1, X + ns * ERS_CTRL_FEATURES);
        T[2 * ns] = t[0];
        T[2 * ns + 1] = t[1];
      }
      ++ns;
    }
  }
  if (count) *count = (int32_t)std::min<int64_t>(ns, INT32_MAX);
  return ERS_OK;
}

ers_status ers_batch_ctrl_stats(const ers_ctx* c, int64_t* proposals, int64_t* rejected,
                                int64_t* krylov_vectors) {
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group())
    return group_ctrl_stats(const_cast<ers_ctx*>(c), proposals, rejected, krylov_vectors);
  if (proposals) *proposals = c->ctrl_proposals;
  if (rejected) *rejected = c->ctrl_rejected;
  if (krylov_vectors) *krylov_vectors = c->stats.krylov_vectors;
  return ERS_OK;
}

ers_status ers_get_state_inst(const ers_ctx* cc, int32_t k, double* t, double* x, double* h) {
  ers_ctx* c = const_cast<ers_ctx*>(cc);
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group()) return group_get_state_inst(c, k, t, x, h);
  DeviceGuard dg(c->device);
  if (k < 0 || k >= c->ninst) return ctx_fail(c, ERS_ERR_INVALID, "instance index out of range");
  if (c->bks) {
    if (t) *t = c->t_inst[k];
    if (h) *h = c->hprop_inst[k];
  } else {
    if (t) *t = c->t;
    if (h) *h = c->h;
  }
  if (x) {
    int lo = c->orig_off.empty() ? 0 : c->orig_off[k];
    int hi = c->orig_off.empty() ? c->n : c->orig_off[k + 1];
    std::vector<double> xp(c->n);
    BCU(cudaMemcpyAsync(xp.data(), c->x, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
    BCU(cudaStreamSynchronize(c->stream));
    for (int v = lo; v < hi; ++v) x[v - lo] = xp[c->sym.iperm[v]];
  }
  return ERS_OK;
}

}  // extern "C"
