// Sparse matrix-vector products and the supernodal triangular solves with the factors
// of G_k (Algorithm 1: "Solve -G w = C v_j"; Alg. 2's setup solves).
//
// The solves are persistent and sync-free.  A CTA takes the next entry of a topologically
// ordered work list (atomic counter), stages the entry's factor data in shared memory
// BEFORE waiting on its dependency word (bounded spin), then runs it and publishes
// completion.  Entries only wait on earlier entries, so the scheme cannot deadlock.
//   GROUP: up to 8 small supernodes, one per warp (diagonal block + all rows);
//   DIAG : a large supernode's diagonal block and its nearest row chunk (the rows of the
//          next supernode up the tree), done by the whole CTA, so a chain of separator
//          supernodes hands off once per link;
//   OFF  : a further row chunk of a large supernode.
//   forward  (L y = b):  a supernode starts once every unit scattering into its rows is
//                        done; y_s <- L11^-1 y_s; y_R -= L21 y_s (FP64 atomics); the unit
//                        then bumps the arrival counter of every supernode it touched.
//   backward (U x = y):  the rows R_off of a supernode lie on its path to the root and a
//                        supernode finishes only after its parent, so a unit waits for the
//                        lowest supernode its rows touch; x_s <- U11^-1 (y_s - U12 x_R).
// NRHS right-hand sides (stride n) share each pass over the factors.
#include <mutex>
#include <string>

#include "ers_internal.h"
#include "kcommon.cuh"

namespace ers {

constexpr int SOLVE_THREADS = 256;
constexpr int UNR = 8;           // independent loads per batch in the warp tasks
constexpr int CHB = 64;          // rows of a CTA chunk (matches SymbolicOptions::solve_chunk)
constexpr int LDP = CHB + 1;     // padded leading dimension of a staged panel (no bank conflicts)

// y = A x for a CSR matrix with short rows
__global__ void k_spmv(int nrows, const int32_t* ptr, const int32_t* idx, const double* val,
                       const double* x, double* y, double alpha) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  double acc = 0.0;
  for (int e = ptr[i]; e < ptr[i + 1]; ++e) acc += val[e] * x[idx[e]];
  y[i] = alpha * acc;
}

struct SolveArgs {
  DevicePlan P;
  double* y;        // nrhs vectors, stride n (in place)
  int n;
  unsigned* status;
  double* Z;        // merged blocks: z = M_L y (forward result), accumulates y - U12 x_R
  double* part;     // partial sums of MGEMV tasks: slot x 64 x MAX_RHS
  const int* done[MAX_RHS];   // Arnoldi solves: the spaces' done flags (ndone of them)
  int ndone;
};

// An Arnoldi solve whose spaces have all finished does nothing (the host learns of it with
// a lag and may have launched it already).  Uniform over the grid: the flags were written by
// earlier launches.
__device__ __forceinline__ bool solve_skipped(const SolveArgs& A) {
  if (A.ndone == 0) return false;
  __shared__ int s_skip;
  if (threadIdx.x == 0) {
    int all = 1;
    for (int b = 0; b < A.ndone; ++b) all &= __ldcg(A.done[b]) != 0;
    s_skip = all;
  }
  __syncthreads();
  return s_skip != 0;
}

// shared-memory layout of a CTA (doubles)
constexpr int SM_D = 64 * 64;            // diagonal block
constexpr int SM_P = LDP * 64;           // panel chunk, column-major with ld LDP
constexpr int SM_V = MAX_RHS * 64;       // vectors
constexpr int SM_PART = 4 * 64 * MAX_RHS;
constexpr int SOLVE_SMEM = (SM_D + SM_P + 2 * SM_V + SM_PART) * 8;

// A GROUP entry of k warp tasks gives each of them 1/k of the CTA's shared memory: its vectors
// (SM_V doubles) and a staging area for its supernode's factor values; a self-scheduling warp
// has 1/8 (WARP_SM).
constexpr int CTA_SM = SOLVE_SMEM / 8;
constexpr int WARP_SM = CTA_SM / (SOLVE_THREADS / 32);
__device__ __forceinline__ int group_share(int ntasks) { return (CTA_SM / max(ntasks, 1)) & ~1; }

// Asynchronous 8-byte global -> shared copies (they stay in flight through a dependency wait;
// cp_async_wait_all makes them visible to the issuing lane, a __syncwarp to the warp).
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void warp_stage(double* dst, const double* src, int cnt, int lane) {
  for (int e = lane; e < cnt; e += 32) cp_async8(dst + e, src + e);
}

// factor value at M + off: from shared memory (staged) or through the read-only path
template <bool SMEM>
__device__ __forceinline__ double fval(const double* M, int64_t off) {
  if constexpr (SMEM) return M[off];
  else return __ldg(M + off);
}

// z_q = sum_{j in tri(q)} M[q + j w] y_j for lanes q (lower: j <= q, upper: j >= q)
template <int NRHS, bool LOWER, bool SMEM = false>
__device__ __forceinline__ void warp_tri_gemv(const double* M, int w, const double (*ys)[64],
                                              double (*z)[NRHS], int lane) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int q = lane + 32 * h;
#pragma unroll
    for (int k = 0; k < NRHS; ++k) z[h][k] = 0.0;
    if (q >= w) continue;
    int j0 = LOWER ? 0 : q, j1 = LOWER ? q + 1 : w;
    int j = j0;
    for (; j + UNR <= j1; j += UNR) {
      double m[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) m[u] = fval<SMEM>(M, q + (int64_t)(j + u) * w);
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) z[h][k] += m[u] * ys[k][j + u];
    }
    for (; j < j1; ++j) {
      double m = fval<SMEM>(M, q + (int64_t)j * w);
#pragma unroll
      for (int k = 0; k < NRHS; ++k) z[h][k] += m * ys[k][j];
    }
  }
}

// rows [0, r) of y_R -= L21 z, lanes over rows (L21 column-major r x w, from M)
template <int NRHS, bool SMEM>
__device__ __forceinline__ void fwd_panel(const SolveArgs& A, const double* M, const int32_t* R,
                                          int w, int r, int row0, const double (*ys)[64],
                                          int lane) {
  const int n = A.n;
  for (int i = lane; i < r; i += 32) {
    double acc[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) acc[k] = 0.0;
    int j = 0;
    for (; j + UNR <= w; j += UNR) {
      double l[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) l[u] = fval<SMEM>(M, i + (int64_t)(j + u) * r);
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) acc[k] += l[u] * ys[k][j + u];
    }
    for (; j < w; ++j) {
      const double l = fval<SMEM>(M, i + (int64_t)j * r);
#pragma unroll
      for (int k = 0; k < NRHS; ++k) acc[k] += l * ys[k][j];
    }
    const int row = i < 32 ? row0 : __ldg(R + i);
#pragma unroll
    for (int k = 0; k < NRHS; ++k) atomicAdd(A.y + (int64_t)k * n + row, -acc[k]);
  }
}

// one small supernode, forward, by one warp.  Its factor values (when they fit the warp's
// staging area), first 32 row indices and first 32 targets are requested before the wait on
// its children, so that only the y loads, the FMAs and the scatter follow the hand-off.
template <int NRHS>
__device__ void fwd_small(const SolveArgs& A, const SolveTask& T, int lane, double* region,
                          int cap) {
  const DevicePlan& P = A.P;
  double (*ys)[64] = reinterpret_cast<double (*)[64]>(region);
  double* stg = region + SM_V;
  int32_t* arrive = P.sync + 2;
  const int n = A.n;
  const int s = T.sn, c0 = T.c0, w = T.w, r = T.r;
  const double* Li = P.LDi + T.d_off;
  const double* Lo = P.Lo + T.o_off;
  const int32_t* R = P.rows + T.row_off;
  // staging pays only while the children are still running: a task whose arrivals are all
  // in streams its factor values directly (cap: the region's doubles after the vectors)
  int pending = 0;
  if (lane == 0) pending = ld_acquire(arrive + s) < T.wait_cnt;
  pending = __shfl_sync(0xffffffffu, pending, 0);
  const bool staged = pending && w * w + r * w <= cap;
  if (staged) {
    warp_stage(stg, Li, w * w, lane);
    warp_stage(stg + w * w, Lo, r * w, lane);
  }
  const int row0 = lane < r ? __ldg(R + lane) : 0;
  const int tgt0 = lane < T.ntgt ? __ldg(P.fwd_tgt + T.tgt0 + lane) : 0;
  int ok = 1;
  if (lane == 0 && pending) ok = wait_geq(arrive + s, T.wait_cnt, A.status);   // else seen
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) { cp_async_wait_all(); __syncwarp(); return; }
  __threadfence();
  for (int q = lane; q < w; q += 32)
#pragma unroll
    for (int k = 0; k < NRHS; ++k) ys[k][q] = __ldcg(A.y + (int64_t)k * n + c0 + q);
  cp_async_wait_all();
  __syncwarp();
  double z[2][NRHS];
  if (staged) warp_tri_gemv<NRHS, true, true>(stg, w, ys, z, lane);
  else warp_tri_gemv<NRHS, true, false>(Li, w, ys, z, lane);
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int q = lane + 32 * h;
    if (q < w)
#pragma unroll
      for (int k = 0; k < NRHS; ++k) {
        ys[k][q] = z[h][k];
        A.y[(int64_t)k * n + c0 + q] = z[h][k];
      }
  }
  __syncwarp();
  if (staged) fwd_panel<NRHS, true>(A, stg + w * w, R, w, r, row0, ys, lane);
  else fwd_panel<NRHS, false>(A, Lo, R, w, r, row0, ys, lane);
  __threadfence();
  __syncwarp();
  // one lane per target: every lane's scatter is ordered before the barrier above
  for (int q = lane; q < T.ntgt; q += 32)
    red_release_add(arrive + (q < 32 ? tgt0 : __ldg(P.fwd_tgt + T.tgt0 + q)), 1);
  __syncwarp();
}

// Cross-lane sums of 8 per-lane accumulators: lane i holds p[c] (its rows' contribution to
// column cb + c); a recursive-halving exchange over lane bits 2..0 (each step keeps half of
// the columns and adds the partner's half) leaves the sum over 8 lanes of column
// cb + (lane & 7) in p[0], and xors over bits 3 and 4 add the other 24 lanes: 9 adds and
// 9 shuffles for 8 columns, once per column block after the FMAs of all its rows.
__device__ __forceinline__ double warp_reduce8(double (&p)[8], int lane) {
#pragma unroll
  for (int off = 4; off >= 1; off >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int c = 0; c < off; ++c) {
      const double send = upper ? p[c] : p[c + off];
      const double keep = upper ? p[c + off] : p[c];
      p[c] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  double v = p[0] + __shfl_xor_sync(0xffffffffu, p[0], 8);
  return v + __shfl_xor_sync(0xffffffffu, v, 16);
}

// Column sums over the slabs of 32 rows a warp owns, lanes over rows (coalesced panel loads):
// out[k] on lane l = sum_i U[i, cb + (l & 7)] x_i[k] over rows i = i0 + lane + 32 q < i1,
// q < MAXSLAB; FMAs per row, one warp_reduce8 per right-hand side.
template <int NRHS, int MAXSLAB, bool SMEM = false>
__device__ __forceinline__ void warp_colsum8(const double* U, int64_t ld, int cb, int ncols,
                                             int i0, int i1, const double (&xr)[MAXSLAB][NRHS],
                                             double (&out)[NRHS], int lane) {
  double acc[NRHS][8];
#pragma unroll
  for (int k = 0; k < NRHS; ++k)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[k][c] = 0.0;
#pragma unroll
  for (int q = 0; q < MAXSLAB; ++q) {
    const int i = i0 + lane + 32 * q;
    if (i0 + 32 * q >= i1) break;
    const bool act = i < i1;
    const double* urow = U + i + (int64_t)cb * ld;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double u = (act && c < ncols) ? fval<SMEM>(urow, (int64_t)c * ld) : 0.0;
#pragma unroll
      for (int k = 0; k < NRHS; ++k) acc[k][c] = fma(u, xr[q][k], acc[k][c]);
    }
  }
#pragma unroll
  for (int k = 0; k < NRHS; ++k) out[k] = warp_reduce8(acc[k], lane);
}

// one small supernode, backward, by one warp: xs = y_s - U12 x_R with lanes over the rows R
// (8-column sums by warp_colsum8), then x_s = U11^-1 xs.  Before the wait on the parent it
// requests what the parent does not write: the factor values (staged when they fit), the
// first 64 row indices and y_s (only this task writes y_s in the backward pass).
template <int NRHS>
__device__ void bwd_small(const SolveArgs& A, const SolveTask& T, int lane, double* region,
                          int cap) {
  const DevicePlan& P = A.P;
  double (*xs)[64] = reinterpret_cast<double (*)[64]>(region);
  double* stg = region + SM_V;
  int32_t* done = P.sync + 2 + P.nsn;
  const int n = A.n;
  const int s = T.sn, c0 = T.c0, w = T.w, r = T.r;
  const double* Ui = P.UDi + T.d_off;
  const double* Uo = P.Uo + T.o_off;
  const int32_t* R = P.rows + T.row_off;
  // staging pays only while the parent is still running (cap: the region's doubles after
  // the vectors)
  int pending = 0;
  if (lane == 0) pending = T.wait_sn >= 0 && ld_acquire(done + T.wait_sn) < 2;
  pending = __shfl_sync(0xffffffffu, pending, 0);
  const bool staged = pending && w * w + r * w <= cap;
  if (staged) {
    warp_stage(stg, Ui, w * w, lane);
    warp_stage(stg + w * w, Uo, r * w, lane);
  }
  int rowq[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int i = lane + 32 * q;
    rowq[q] = i < r ? __ldg(R + i) : 0;
  }
  for (int q = lane; q < w; q += 32)
#pragma unroll
    for (int k = 0; k < NRHS; ++k) xs[k][q] = __ldcg(A.y + (int64_t)k * n + c0 + q);
  int ok = 1;
  if (lane == 0 && pending) ok = wait_geq(done + T.wait_sn, 2, A.status);   // else seen
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) { cp_async_wait_all(); __syncwarp(); return; }
  __threadfence();
  cp_async_wait_all();
  __syncwarp();
  const double* U = staged ? stg + w * w : Uo;
  // column sums, 64 rows at a time (x of the rows in registers), 8 columns per block
  for (int i0 = 0; i0 < r; i0 += 64) {
    double xr[2][NRHS];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = i0 + lane + 32 * q;
      const bool act = i < r;
      const int row = i0 == 0 ? rowq[q] : (act ? __ldg(R + i) : 0);
#pragma unroll
      for (int k = 0; k < NRHS; ++k) xr[q][k] = act ? __ldcg(A.y + (int64_t)k * n + row) : 0.0;
    }
    for (int cb = 0; cb < w; cb += 8) {
      double v[NRHS];
      if (staged)
        warp_colsum8<NRHS, 2, true>(U, r, cb, min(8, w - cb), i0, min(r, i0 + 64), xr, v, lane);
      else
        warp_colsum8<NRHS, 2, false>(U, r, cb, min(8, w - cb), i0, min(r, i0 + 64), xr, v, lane);
      if (lane < 8 && cb + lane < w)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) xs[k][cb + lane] -= v[k];
      __syncwarp();
    }
  }
  __syncwarp();
  double z[2][NRHS];
  if (staged) warp_tri_gemv<NRHS, false, true>(stg, w, xs, z, lane);
  else warp_tri_gemv<NRHS, false, false>(Ui, w, xs, z, lane);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int q = lane + 32 * h;
    if (q < w)
#pragma unroll
      for (int k = 0; k < NRHS; ++k) A.y[(int64_t)k * n + c0 + q] = z[h][k];
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) st_release(done + s, 2);
  __syncwarp();
}

// Narrow supernodes (w <= LANE_W columns) of one level, forward, one per lane (up to 32 per
// warp task): wait for the lane's own arrivals, y_s <- L11^-1 y_s, y_R -= L21 y_s, then
// arrive at the targets.
constexpr int LANE_W = 4;
template <int NRHS>
__device__ __noinline__ void fwd_lanes(const SolveArgs& A, const SolveTask& T, int lane) {
  const DevicePlan& P = A.P;
  int32_t* arrive = P.sync + 2;
  const int n = A.n;
  if (lane < T.r0) {
    const int4 it = __ldg(reinterpret_cast<const int4*>(P.fwd_lane) + T.sn + lane);
    const int s = it.x;
    const int c0 = __ldg(P.sn_start + s), w = __ldg(P.sn_start + s + 1) - c0;
    const int64_t rp = __ldg(P.rptr + s);
    const int r = (int)(__ldg(P.rptr + s + 1) - rp);
    const double* Li = P.LDi + __ldg(P.d_off + s);
    const double* Lo = P.Lo + __ldg(P.o_off + s);
    if (wait_geq(arrive + s, it.w, A.status)) {
      double y[LANE_W][NRHS], z[LANE_W][NRHS];
#pragma unroll
      for (int j = 0; j < LANE_W; ++j)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          y[j][k] = j < w ? __ldcg(A.y + (int64_t)k * n + c0 + j) : 0.0;
          z[j][k] = 0.0;
        }
      // z = L11^-1 y (lower triangular, column-major w x w)
#pragma unroll
      for (int q = 0; q < LANE_W; ++q)
#pragma unroll
        for (int j = 0; j <= q; ++j)
          if (q < w) {
            const double m = __ldg(Li + q + j * w);
#pragma unroll
            for (int k = 0; k < NRHS; ++k) z[q][k] += m * y[j][k];
          }
#pragma unroll
      for (int q = 0; q < LANE_W; ++q)
        if (q < w)
#pragma unroll
          for (int k = 0; k < NRHS; ++k) A.y[(int64_t)k * n + c0 + q] = z[q][k];
      for (int i = 0; i < r; ++i) {
        double acc[NRHS];
#pragma unroll
        for (int k = 0; k < NRHS; ++k) acc[k] = 0.0;
#pragma unroll
        for (int j = 0; j < LANE_W; ++j)
          if (j < w) {
            const double l = __ldg(Lo + i + (int64_t)j * r);
#pragma unroll
            for (int k = 0; k < NRHS; ++k) acc[k] += l * z[j][k];
          }
        const int row = __ldg(P.rows + rp + i);
#pragma unroll
        for (int k = 0; k < NRHS; ++k) atomicAdd(A.y + (int64_t)k * n + row, -acc[k]);
      }
      __threadfence();
      for (int q = 0; q < it.z; ++q) red_release_add(arrive + __ldg(P.fwd_tgt + it.y + q), 1);
    }
  }
  __syncwarp();
}

// Narrow supernodes of one depth, backward, one per lane: once the parent is done,
// x_s = U11^-1 (y_s - U12 x_R); then the supernode is marked done for its children.
template <int NRHS>
__device__ __noinline__ void bwd_lanes(const SolveArgs& A, const SolveTask& T, int lane) {
  const DevicePlan& P = A.P;
  int32_t* done = P.sync + 2 + P.nsn;
  const int n = A.n;
  if (lane < T.r0) {
    const int4 it = __ldg(reinterpret_cast<const int4*>(P.bwd_lane) + T.sn + lane);
    const int s = it.x, parent = it.y;
    const int c0 = __ldg(P.sn_start + s), w = __ldg(P.sn_start + s + 1) - c0;
    const int64_t rp = __ldg(P.rptr + s);
    const int r = (int)(__ldg(P.rptr + s + 1) - rp);
    const double* Ui = P.UDi + __ldg(P.d_off + s);
    const double* Uo = P.Uo + __ldg(P.o_off + s);
    if (parent < 0 || wait_geq(done + parent, 2, A.status)) {
      double acc[LANE_W][NRHS];
#pragma unroll
      for (int j = 0; j < LANE_W; ++j)
#pragma unroll
        for (int k = 0; k < NRHS; ++k)
          acc[j][k] = j < w ? __ldcg(A.y + (int64_t)k * n + c0 + j) : 0.0;
      for (int i = 0; i < r; ++i) {
        const int row = __ldg(P.rows + rp + i);
        double xr[NRHS];
#pragma unroll
        for (int k = 0; k < NRHS; ++k) xr[k] = __ldcg(A.y + (int64_t)k * n + row);
#pragma unroll
        for (int j = 0; j < LANE_W; ++j)
          if (j < w) {
            const double u = __ldg(Uo + i + (int64_t)j * r);
#pragma unroll
            for (int k = 0; k < NRHS; ++k) acc[j][k] -= u * xr[k];
          }
      }
      // x = U11^-1 acc (upper triangular, column-major w x w)
#pragma unroll
      for (int q = 0; q < LANE_W; ++q)
        if (q < w) {
          double x[NRHS];
#pragma unroll
          for (int k = 0; k < NRHS; ++k) x[k] = 0.0;
#pragma unroll
          for (int j = q; j < LANE_W; ++j)
            if (j < w) {
              const double m = __ldg(Ui + q + j * w);
#pragma unroll
              for (int k = 0; k < NRHS; ++k) x[k] += m * acc[j][k];
            }
#pragma unroll
          for (int k = 0; k < NRHS; ++k) A.y[(int64_t)k * n + c0 + q] = x[k];
        }
      __threadfence();
      st_release(done + s, 2);
    }
  }
  __syncwarp();
}

// a far chunk of a large supernode, forward, one warp: lanes over rows,
// y[R[i]] -= sum_j Lo[i + j r] z_j with z = y_s (written by the supernode's DIAG task)
template <int NRHS>
__device__ void fwd_chunk(const SolveArgs& A, const SolveTask& T, int lane, double* buf) {
  const DevicePlan& P = A.P;
  int32_t* arrive = P.sync + 2;
  int32_t* ready = P.sync + 2 + P.nsn;
  const int n = A.n;
  const int s = T.sn, c0 = T.c0, w = T.w, r = T.r;
  const double* Lo = P.Lo + T.o_off;
  const int32_t* R = P.rows + T.row_off;
  double (*zs)[64] = reinterpret_cast<double (*)[64]>(buf);
  const int i = T.r0 + lane;
  const bool act = i < T.r1;
  const int row = act ? __ldg(R + i) : 0;
  int ok = 1;
  if (lane == 0) ok = wait_geq(ready + s, 1, A.status);
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return;
  __threadfence();
  const double* zsrc = T.grp >= 0 ? A.Z : A.y;   // a merged piece's z lives in Z
  for (int q = lane; q < w; q += 32)
#pragma unroll
    for (int k = 0; k < NRHS; ++k) zs[k][q] = __ldcg(zsrc + (int64_t)k * n + c0 + q);
  __syncwarp();
  double acc[NRHS];
#pragma unroll
  for (int k = 0; k < NRHS; ++k) acc[k] = 0.0;
  const double* col = Lo + i;
  constexpr int B = 16;
  for (int j0 = 0; j0 < w; j0 += B) {
    double l[B];
#pragma unroll
    for (int u = 0; u < B; ++u) l[u] = (act && j0 + u < w) ? __ldg(col + (int64_t)(j0 + u) * r) : 0.0;
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (j0 + u < w)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) acc[k] += l[u] * zs[k][j0 + u];
  }
  if (act)
#pragma unroll
    for (int k = 0; k < NRHS; ++k) atomicAdd(A.y + (int64_t)k * n + row, -acc[k]);
  __threadfence();
  __syncwarp();
  if (lane == 0)
    for (int q = 0; q < T.ntgt; ++q) red_release_add(arrive + P.fwd_tgt[T.tgt0 + q], 1);
  __syncwarp();
}

// a far chunk, backward, one warp: y[c0 + j] -= sum_{i in chunk} Uo[i + j r] x[R[i]] over up
// to BCH rows, lanes over rows (coalesced panel loads), FMAs over the chunk's slabs and one
// 8-column exchange per block (warp_colsum8)
constexpr int BCH = 128;         // rows of a backward far chunk (SymbolicOptions::bwd_chunk)
template <int NRHS>
__device__ void bwd_chunk(const SolveArgs& A, const SolveTask& T, int lane, double* buf) {
  const DevicePlan& P = A.P;
  int32_t* done = P.sync + 2 + P.nsn;
  int32_t* arriveb = P.sync + 2 + 2 * P.nsn;
  const int n = A.n;
  const int s = T.sn, c0 = T.c0, w = T.w, r = T.r;
  const double* Uo = P.Uo + T.o_off;
  const int32_t* R = P.rows + T.row_off;
  (void)buf;
  int ok = 1;
  if (lane == 0) ok = wait_geq(done + T.wait_sn, 2, A.status);
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return;
  __threadfence();
  double xr[BCH / 32][NRHS];      // x at the chunk's rows: row T.r0 + lane + 32 q
#pragma unroll
  for (int q = 0; q < BCH / 32; ++q) {
    const int i = T.r0 + lane + 32 * q;
    const bool act = i < T.r1;
    const int row = act ? __ldg(R + i) : 0;
#pragma unroll
    for (int k = 0; k < NRHS; ++k) xr[q][k] = act ? __ldcg(A.y + (int64_t)k * n + row) : 0.0;
  }
  double* dst = T.grp >= 0 ? A.Z : A.y;   // a merged piece accumulates in Z
  for (int cb = 0; cb < w; cb += 8) {
    double v[NRHS];
    warp_colsum8<NRHS, BCH / 32>(Uo, r, cb, min(8, w - cb), T.r0, T.r1, xr, v, lane);
    if (lane < 8 && cb + lane < w)
#pragma unroll
      for (int k = 0; k < NRHS; ++k) atomicAdd(dst + (int64_t)k * n + c0 + cb + lane, -v[k]);
  }
  __threadfence();
  __syncwarp();
  if (lane == 0) red_release_add(arriveb + s, 1);
  __syncwarp();
}

// Stage a w x w diagonal block and panel rows [r0, r1) (ld r) into shared memory.  Every
// thread first issues all its loads (at most 16 + 16 independent requests), then stores.
__device__ __forceinline__ void stage(const double* D, int w, const double* Pn, int r, int r0,
                                      int r1, double* sD, double* sP, bool with_diag) {
  const int tid = threadIdx.x;
  constexpr int PER = (64 * 64) / SOLVE_THREADS;   // 16
  const int rows = r1 - r0;
  const int nd = with_diag ? w * w : 0, np = rows * w;
  double vd[PER], vp[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    int e = tid + u * SOLVE_THREADS;
    vd[u] = e < nd ? __ldg(D + e) : 0.0;
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    int e = tid + u * SOLVE_THREADS;
    int i = e % max(rows, 1), j = e / max(rows, 1);
    vp[u] = e < np ? __ldg(Pn + r0 + i + (int64_t)j * r) : 0.0;
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    int e = tid + u * SOLVE_THREADS;
    if (e < nd) sD[e] = vd[u];
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    int e = tid + u * SOLVE_THREADS;
    int i = e % max(rows, 1), j = e / max(rows, 1);
    if (e < np) sP[i + j * LDP] = vp[u];
  }
}

// One row tile of a merged block times a column range of its explicit inverse (a CTA
// entry).  Forward: partial = M_L[rows of piece sn, columns r0..r1-1] y once the arrivals at
// those column pieces are complete; backward: partial = M_U[...] Z once their far chunks have
// subtracted U12 x_R.  The partial goes to the task's slot; the last task of the row tile
// sums the tile's slots in slot order (a fixed order, so the result is deterministic) and
// writes z into Z (forward: then the piece is ready for its far chunks) or x into y
// (backward: the block's pieces complete together once all its row tiles are written, so no
// piece completes before its parent).
constexpr int MG_COLS = 512;     // columns of one MGEMV task (merge_col_block x 64 at most)
template <int NRHS>
__device__ void mgemv(const SolveArgs& A, const SolveTask& T, double* sm, bool fwd) {
  const DevicePlan& P = A.P;
  const int nsn = P.nsn, n = A.n;
  int32_t* arrive = P.sync + 2;
  int32_t* flag = P.sync + 2 + nsn;             // forward ready (1) / backward done (2)
  int32_t* arriveb = P.sync + 2 + 2 * nsn;
  int32_t* tilecnt = P.sync + 2 + (fwd ? 3 : 4) * (size_t)nsn;
  int32_t* grpcnt = P.sync + 2 + 5 * (size_t)nsn;
  const int tid = threadIdx.x, lane = tid & 31;
  const int ncol = (int)(T.row_off - T.o_off);
  double* vs = sm;                              // [NRHS][MG_COLS]
  double* part = sm + NRHS * MG_COLS;           // [4][64][NRHS]
  __shared__ int s_ok, s_last;
  if (tid < 32) {
    const int j = T.r0 + lane;
    int ok = 1;
    if (j < T.r1)
      ok = fwd ? wait_geq(arrive + j, __ldg(P.fwd_expect + j), A.status)
               : wait_geq(arriveb + j, __ldg(P.bwd_nchunk + j), A.status);
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return;
  __threadfence();
  const double* src = fwd ? A.y : A.Z;
  for (int e = tid; e < ncol * NRHS; e += SOLVE_THREADS) {
    const int k = e / ncol, c = e - k * ncol;
    vs[k * MG_COLS + c] = __ldcg(src + (int64_t)k * n + T.o_off + c);
  }
  __syncthreads();
  const int q = tid & 63, g = tid >> 6;         // row of the tile, column group (c = g mod 4)
  const double* M = (fwd ? P.ML : P.MU) + T.d_off;
  const int64_t ld = T.r;
  double acc[NRHS];
#pragma unroll
  for (int k = 0; k < NRHS; ++k) acc[k] = 0.0;
  if (q < T.w) {
    const double* mq = M + q;
    int c = g;
    for (; c + 28 < ncol; c += 32) {            // 8 independent loads per thread
      double m[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) m[u] = __ldg(mq + (int64_t)(c + 4 * u) * ld);
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) acc[k] += m[u] * vs[k * MG_COLS + c + 4 * u];
    }
    for (; c < ncol; c += 4) {
      const double m = __ldg(mq + (int64_t)c * ld);
#pragma unroll
      for (int k = 0; k < NRHS; ++k) acc[k] += m * vs[k * MG_COLS + c];
    }
  }
#pragma unroll
  for (int k = 0; k < NRHS; ++k) part[(g * 64 + q) * NRHS + k] = acc[k];
  __syncthreads();
  if (tid < T.w) {
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      const double v = part[(0 * 64 + tid) * NRHS + k] + part[(1 * 64 + tid) * NRHS + k] +
                       part[(2 * 64 + tid) * NRHS + k] + part[(3 * 64 + tid) * NRHS + k];
      A.part[((int64_t)T.tgt0 * 64 + tid) * MAX_RHS + k] = v;
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(tilecnt + T.sn, 1) == T.wait_cnt - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < T.w) {
    double* dst = fwd ? A.Z : A.y;
#pragma unroll
    for (int k = 0; k < NRHS; ++k) {
      double z = 0.0;
      for (int t = 0; t < T.wait_cnt; ++t)
        z += __ldcg(A.part + ((int64_t)(T.wait_sn + t) * 64 + tid) * MAX_RHS + k);
      dst[(int64_t)k * n + T.c0 + tid] = z;
    }
  }
  __threadfence();
  __syncthreads();
  if (fwd) {
    if (tid == 0) st_release(flag + T.sn, 1);
    return;
  }
  if (tid < 32) {
    const int f = __ldg(P.grp_first + T.grp), l = __ldg(P.grp_last + T.grp);
    int all = 0;
    if (lane == 0) all = atomicAdd(grpcnt + f, 1) == l - f;
    all = __shfl_sync(0xffffffffu, all, 0);
    if (all) {
      __threadfence();
      for (int s2 = f + lane; s2 <= l; s2 += 32) st_release(flag + s2, 2);
    }
  }
}

// Work lists made of warp tasks only (tree-structured factors: chains, batches of chains):
// every warp schedules itself over the flattened list (entries in order, each entry's tasks
// in order, so still topological), with the next index fetched while the current task runs.
// No CTA barrier is involved, so a warp whose task is done does not wait for the slowest warp
// of its CTA.  Deadlock-free like the CTA list: a warp holds at most its current task and
// the next one, and the smallest unfinished task is always being run.
template <int NRHS, bool FWD>
__device__ __forceinline__ void warp_scheduled(const SolveArgs& A, double* sm, int wq, int lane) {
  const DevicePlan& P = A.P;
  int32_t* ctr = P.sync + (FWD ? 0 : 1);
  const SolveTask* list = FWD ? P.fwd_warp : P.bwd_warp;
  const int N = FWD ? P.nfwd_warp : P.nbwd_warp;
  double* region = sm + wq * WARP_SM;
  int k = 0, nk = 0;
  if (lane == 0) k = atomicAdd(ctr, 1);
  k = __shfl_sync(0xffffffffu, k, 0);
  while (k < N) {
    if (lane == 0) nk = atomicAdd(ctr, 1);
    const SolveTask& U = list[k];
    if (FWD) {
      if (U.kind == TASK_LANES) fwd_lanes<NRHS>(A, U, lane);
      else fwd_small<NRHS>(A, U, lane, region, WARP_SM - SM_V);
    } else {
      if (U.kind == TASK_LANES) bwd_lanes<NRHS>(A, U, lane);
      else bwd_small<NRHS>(A, U, lane, region, WARP_SM - SM_V);
    }
    k = __shfl_sync(0xffffffffu, nk, 0);
  }
}

// The same loop out of line.  The CTA-list kernels come in two variants, without (OOL =
// false) and with a call of it on their entry path (never taken for their lists): ptxas
// allocates their registers differently, and which variant is faster depends on the work
// list (one is 30 % faster on the 32 x 32 mesh, the other 7 % faster on the 100^3 mesh), so
// the autotuner times both.
template <int NRHS, bool FWD>
__device__ __noinline__ void warp_scheduled_ool(const SolveArgs& A, double* sm, int wq, int lane) {
  warp_scheduled<NRHS, FWD>(A, sm, wq, lane);
}

// MINB: resident CTAs per SM the kernel is compiled for (register cap 65536 / (256 MINB)); the
// launch uses the instance matching the autotuned count, so no count pays the tighter cap.
template <int NRHS, int MINB, bool OOL>
__global__ void __launch_bounds__(SOLVE_THREADS, MINB) k_trsv_fwd(SolveArgs A) {
  extern __shared__ double sm[];
  double* sD = sm;
  double* sP = sD + SM_D;
  double (*ys)[64] = reinterpret_cast<double (*)[64]>(sP + SM_P);
  double (*zs)[64] = reinterpret_cast<double (*)[64]>(sP + SM_P + SM_V);
  double* part = sP + SM_P + 2 * SM_V;   // [4][64][NRHS]
  __shared__ int s_cur, s_ok;
  const DevicePlan& P = A.P;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  int32_t* sync = P.sync;
  int32_t* arrive = sync + 2;
  int32_t* ready = sync + 2 + P.nsn;
  const int n = A.n;
  if (solve_skipped(A)) return;
  if constexpr (OOL) {
    if (P.nfwd_warp > 0) {
      warp_scheduled_ool<NRHS, true>(A, sm, threadIdx.x >> 5, threadIdx.x & 31);
      return;
    }
  }
  while (true) {
    __syncthreads();
    if (tid == 0) s_cur = atomicAdd(sync, 1);
    __syncthreads();
    int e = s_cur;
    if (e >= P.nfwd) break;
    SolveTask T = P.fwd[e];
    if (T.kind == TASK_GROUP) {
      if (wq < T.r0) {
        const SolveTask& U = P.fwd_small[T.sn + wq];
        if (U.kind == TASK_LANES) fwd_lanes<NRHS>(A, U, lane);
        else {
          const int share = group_share(T.r0);
          fwd_small<NRHS>(A, U, lane, sm + wq * share, share - SM_V);
        }
      }
      continue;
    }
    if (T.kind == TASK_BULK) {
      if (wq < T.r0) fwd_chunk<NRHS>(A, P.fwd_small[T.sn + wq], lane, sm + wq * MAX_RHS * 64);
      continue;
    }
    if (T.kind == TASK_MGEMV) {
      mgemv<NRHS>(A, T, sm, true);
      continue;
    }
    const int s = T.sn, c0 = T.c0, w = T.w, r = T.r;
    const int32_t* R = P.rows + T.row_off;
    bool diag = T.kind == TASK_DIAG;
    stage(P.LDi + T.d_off, w, P.Lo + T.o_off, r, T.r0, T.r1, sD, sP, diag);
    if (tid == 0)
      s_ok = diag ? wait_geq(arrive + s, T.wait_cnt, A.status) : wait_geq(ready + s, 1, A.status);
    __syncthreads();
    if (!s_ok) continue;
    __threadfence();
    if (tid < w)
#pragma unroll
      for (int k = 0; k < NRHS; ++k) ys[k][tid] = __ldcg(A.y + (int64_t)k * n + c0 + tid);
    __syncthreads();
    const int q = tid & 63, g = tid >> 6;   // row / column-group of the 64 x 4 thread grid
    if (diag) {
      // z = L11^-1 y_s, columns split in 4 groups of 16
      double acc[NRHS];
#pragma unroll
      for (int k = 0; k < NRHS; ++k) acc[k] = 0.0;
      if (q < w) {
        int j1 = min(16 * g + 16, q + 1);
        for (int j = 16 * g; j < j1; ++j) {
          double m = sD[q + j * w];
#pragma unroll
          for (int k = 0; k < NRHS; ++k) acc[k] += m * ys[k][j];
        }
      }
#pragma unroll
      for (int k = 0; k < NRHS; ++k) part[(g * 64 + q) * NRHS + k] = acc[k];
      __syncthreads();
      if (tid < w)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          double z = part[(0 * 64 + tid) * NRHS + k] + part[(1 * 64 + tid) * NRHS + k] +
                     part[(2 * 64 + tid) * NRHS + k] + part[(3 * 64 + tid) * NRHS + k];
          zs[k][tid] = z;
          A.y[(int64_t)k * n + c0 + tid] = z;
        }
      __syncthreads();
    } else {
      if (tid < w)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) zs[k][tid] = ys[k][tid];
      __syncthreads();
    }
    // chunk rows [r0, r1): y[R[i]] -= sum_j Lo[i + j r] z_j
    int rows = T.r1 - T.r0;
    {
      double acc[NRHS];
#pragma unroll
      for (int k = 0; k < NRHS; ++k) acc[k] = 0.0;
      if (q < rows) {
        int j1 = min(16 * g + 16, w);
        for (int j = 16 * g; j < j1; ++j) {
          double l = sP[q + j * LDP];
#pragma unroll
          for (int k = 0; k < NRHS; ++k) acc[k] += l * zs[k][j];
        }
      }
#pragma unroll
      for (int k = 0; k < NRHS; ++k) part[(g * 64 + q) * NRHS + k] = acc[k];
    }
    __syncthreads();
    if (tid < rows) {
      int row = __ldg(R + T.r0 + tid);
#pragma unroll
      for (int k = 0; k < NRHS; ++k) {
        double v = part[(0 * 64 + tid) * NRHS + k] + part[(1 * 64 + tid) * NRHS + k] +
                   part[(2 * 64 + tid) * NRHS + k] + part[(3 * 64 + tid) * NRHS + k];
        atomicAdd(A.y + (int64_t)k * n + row, -v);
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      if (diag) st_release(ready + s, 1);
      for (int t = 0; t < T.ntgt; ++t) red_release_add(arrive + P.fwd_tgt[T.tgt0 + t], 1);
    }
  }
}

template <int NRHS, int MINB, bool OOL>
__global__ void __launch_bounds__(SOLVE_THREADS, MINB) k_trsv_bwd(SolveArgs A) {
  extern __shared__ double sm[];
  double* sD = sm;
  double* sP = sD + SM_D;
  double (*xr)[64] = reinterpret_cast<double (*)[64]>(sP + SM_P);          // x at chunk rows
  double (*xs)[64] = reinterpret_cast<double (*)[64]>(sP + SM_P + SM_V);   // x_s
  double* part = sP + SM_P + 2 * SM_V;
  __shared__ int s_cur, s_ok;
  const DevicePlan& P = A.P;
  const int tid = threadIdx.x, lane = tid & 31, wq = tid >> 5;
  int32_t* sync = P.sync;
  int32_t* done = sync + 2 + P.nsn;
  int32_t* arriveb = sync + 2 + 2 * P.nsn;
  const int n = A.n;
  if (solve_skipped(A)) return;
  if constexpr (OOL) {
    if (P.nbwd_warp > 0) {
      warp_scheduled_ool<NRHS, false>(A, sm, threadIdx.x >> 5, threadIdx.x & 31);
      return;
    }
  }
  while (true) {
    __syncthreads();
    if (tid == 0) s_cur = atomicAdd(sync + 1, 1);
    __syncthreads();
    int e = s_cur;
    if (e >= P.nbwd) break;
    SolveTask T = P.bwd[e];
    if (T.kind == TASK_GROUP) {
      if (wq < T.r0) {
        const SolveTask& U = P.bwd_small[T.sn + wq];
        if (U.kind == TASK_LANES) bwd_lanes<NRHS>(A, U, lane);
        else {
          const int share = group_share(T.r0);
          bwd_small<NRHS>(A, U, lane, sm + wq * share, share - SM_V);
        }
      }
      continue;
    }
    if (T.kind == TASK_BULK) {
      if (wq < T.r0) bwd_chunk<NRHS>(A, P.bwd_small[T.sn + wq], lane, sm + wq * MAX_RHS * 64);
      continue;
    }
    if (T.kind == TASK_MGEMV) {
      mgemv<NRHS>(A, T, sm, false);
      continue;
    }
    const int s = T.sn, c0 = T.c0, w = T.w, r = T.r;
    const int32_t* R = P.rows + T.row_off;
    bool diag = T.kind == TASK_DIAG;
    stage(P.UDi + T.d_off, w, P.Uo + T.o_off, r, T.r0, T.r1, sD, sP, diag);
    if (tid == 0) {
      int ok = 1;
      if (T.wait_sn >= 0) ok = wait_geq(done + T.wait_sn, 2, A.status);
      if (ok && diag) ok = wait_geq(arriveb + s, T.wait_cnt, A.status);
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) continue;
    __threadfence();
    int rows = T.r1 - T.r0;
    if (tid < rows) {
      int row = __ldg(R + T.r0 + tid);
#pragma unroll
      for (int k = 0; k < NRHS; ++k) xr[k][tid] = __ldcg(A.y + (int64_t)k * n + row);
    }
    __syncthreads();
    const int q = tid & 63, g = tid >> 6;   // column / row-group of the 64 x 4 thread grid
    {
      double acc[NRHS];
#pragma unroll
      for (int k = 0; k < NRHS; ++k) acc[k] = 0.0;
      if (q < w) {
        int i1 = min(16 * g + 16, rows);
        for (int i = 16 * g; i < i1; ++i) {
          double u = sP[i + q * LDP];
#pragma unroll
          for (int k = 0; k < NRHS; ++k) acc[k] += u * xr[k][i];
        }
      }
#pragma unroll
      for (int k = 0; k < NRHS; ++k) part[(g * 64 + q) * NRHS + k] = acc[k];
    }
    __syncthreads();
    if (!diag) {
      if (tid < w)
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
          double v = part[(0 * 64 + tid) * NRHS + k] + part[(1 * 64 + tid) * NRHS + k] +
                     part[(2 * 64 + tid) * NRHS + k] + part[(3 * 64 + tid) * NRHS + k];
          atomicAdd(A.y + (int64_t)k * n + c0 + tid, -v);
        }
      __threadfence();
      __syncthreads();
      if (tid == 0) red_release_add(arriveb + s, 1);
      continue;
    }
    if (tid < w)
#pragma unroll
      for (int k = 0; k < NRHS; ++k) {
        double v = part[(0 * 64 + tid) * NRHS + k] + part[(1 * 64 + tid) * NRHS + k] +
                   part[(2 * 64 + tid) * NRHS + k] + part[(3 * 64 + tid) * NRHS + k];
        xs[k][tid] = __ldcg(A.y + (int64_t)k * n + c0 + tid) - v;
      }
    __syncthreads();
    // x_s = U11^-1 xs, columns split in 4 groups of 16
    {
      double acc[NRHS];
#pragma unroll
      for (int k = 0; k < NRHS; ++k) acc[k] = 0.0;
      if (q < w) {
        int j0 = max(16 * g, q), j1 = min(16 * g + 16, w);
        for (int j = j0; j < j1; ++j) {
          double m = sD[q + j * w];
#pragma unroll
          for (int k = 0; k < NRHS; ++k) acc[k] += m * xs[k][j];
        }
      }
#pragma unroll
      for (int k = 0; k < NRHS; ++k) part[(g * 64 + q) * NRHS + k] = acc[k];
    }
    __syncthreads();
    if (tid < w)
#pragma unroll
      for (int k = 0; k < NRHS; ++k)
        A.y[(int64_t)k * n + c0 + tid] = part[(0 * 64 + tid) * NRHS + k] +
                                         part[(1 * 64 + tid) * NRHS + k] +
                                         part[(2 * 64 + tid) * NRHS + k] +
                                         part[(3 * 64 + tid) * NRHS + k];
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(done + s, 2);
  }
}

void launch_spmv(ers_ctx* c, const int32_t* ptr, const int32_t* idx, const double* val,
                 const double* x, double* y, double alpha) {
  k_spmv<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->n, ptr, idx, val, x, y, alpha);
  c->stats.kernel_launches++;
}

// Failure-path self-test: one thread waits, with the solves' bounded wait, on a flag that
// nothing sets; the wait gives up after SPIN_LIMIT polls and records ST_TIMEOUT.
__global__ void k_wait_probe(const int32_t* flag, unsigned* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) wait_geq(flag, 1, status);
}

cudaError_t launch_wait_probe(ers_ctx* c, const int32_t* flag) {
  k_wait_probe<<<1, 32, 0, c->stream>>>(flag, c->d_status);
  c->stats.kernel_launches++;
  return cudaGetLastError();
}

// The warp-scheduled passes (a work list of warp tasks only) as kernels of their own, so that
// the CTA-list kernels keep their register allocation.
template <int NRHS, int MINB, bool FWD>
__global__ void __launch_bounds__(SOLVE_THREADS, MINB) k_trsv_warp(SolveArgs A) {
  extern __shared__ double sm[];
  if (solve_skipped(A)) return;
  warp_scheduled<NRHS, FWD>(A, sm, threadIdx.x >> 5, threadIdx.x & 31);
}

template <int NRHS, int MINB>
static void launch_pair_minb(ers_ctx* c, const SolveArgs& A, int blocks) {
  const bool ool = c->solve_variant != 0;
  if (A.P.nfwd_warp > 0 && c->solve_warp_fwd)
    k_trsv_warp<NRHS, MINB, true><<<blocks, SOLVE_THREADS, SOLVE_SMEM, c->stream>>>(A);
  else if (ool)
    k_trsv_fwd<NRHS, MINB, true><<<blocks, SOLVE_THREADS, SOLVE_SMEM, c->stream>>>(A);
  else
    k_trsv_fwd<NRHS, MINB, false><<<blocks, SOLVE_THREADS, SOLVE_SMEM, c->stream>>>(A);
  if (A.P.nbwd_warp > 0 && c->solve_warp_bwd)
    k_trsv_warp<NRHS, MINB, false><<<blocks, SOLVE_THREADS, SOLVE_SMEM, c->stream>>>(A);
  else if (ool)
    k_trsv_bwd<NRHS, MINB, true><<<blocks, SOLVE_THREADS, SOLVE_SMEM, c->stream>>>(A);
  else
    k_trsv_bwd<NRHS, MINB, false><<<blocks, SOLVE_THREADS, SOLVE_SMEM, c->stream>>>(A);
}

template <int NRHS>
static void launch_pair(ers_ctx* c, const SolveArgs& A, int blocks) {
  if (c->solve_ctas_per_sm >= 3) launch_pair_minb<NRHS, 3>(c, A, blocks);
  else launch_pair_minb<NRHS, 2>(c, A, blocks);
}

template <int NRHS, int MINB>
static cudaError_t set_smem_attributes() {
  const void* fns[] = {(const void*)k_trsv_fwd<NRHS, MINB, false>,
                       (const void*)k_trsv_bwd<NRHS, MINB, false>,
                       (const void*)k_trsv_fwd<NRHS, MINB, true>,
                       (const void*)k_trsv_bwd<NRHS, MINB, true>,
                       (const void*)k_trsv_warp<NRHS, MINB, true>,
                       (const void*)k_trsv_warp<NRHS, MINB, false>};
  for (const void* f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, SOLVE_SMEM);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t solve_kernel_attributes() {
  cudaError_t e = set_smem_attributes<1, 2>();
  if (e == cudaSuccess) e = set_smem_attributes<2, 2>();
  if (e == cudaSuccess) e = set_smem_attributes<3, 2>();
  if (e == cudaSuccess) e = set_smem_attributes<1, 3>();
  if (e == cudaSuccess) e = set_smem_attributes<2, 3>();
  if (e == cudaSuccess) e = set_smem_attributes<3, 3>();
  return e;
}

// Solve G_k X = Y in place for nrhs vectors (stride n).  done (ndone device flags, or
// nullptr): the whole pass is skipped on the device when every flag is set.
cudaError_t launch_solve_skip(ers_ctx* c, double* y, int nrhs, const int* const* done, int ndone) {
  DevicePlan& P = c->plan;
  if (nrhs < 1 || nrhs > MAX_RHS) return cudaErrorInvalidValue;
  if (done && (ndone < 1 || ndone > MAX_RHS)) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(P.sync, 0, sizeof(int32_t) * solve_sync_words(P.nsn), c->stream);
  if (e != cudaSuccess) return e;
  SolveArgs A{P, y, c->n, c->d_status, c->solve_z, c->solve_part, {}, 0};
  if (done) {
    for (int b = 0; b < ndone; ++b) A.done[b] = done[b];
    A.ndone = ndone;
  }
  int blocks = c->sm_count * c->solve_ctas_per_sm;
  std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
  if (c->profile) {
    if (c->ev_free.empty()) {
      cudaEventCreate(&ev.first);
      cudaEventCreate(&ev.second);
    } else {
      ev = c->ev_free.back();
      c->ev_free.pop_back();
    }
    cudaEventRecord(ev.first, c->stream);
  }
  if (nrhs == 1) launch_pair<1>(c, A, blocks);
  else if (nrhs == 2) launch_pair<2>(c, A, blocks);
  else launch_pair<3>(c, A, blocks);
  if (c->profile) {
    cudaEventRecord(ev.second, c->stream);
    c->ev_used.push_back(ev);
  }
  c->stats.solves += nrhs;
  c->stats.solve_passes += 1;
  c->stats.solve_rhs += nrhs;
  c->stats.kernel_launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_solve(ers_ctx* c, double* y, int nrhs) { return launch_solve_skip(c, y, nrhs, nullptr, 0); }

}  // namespace ers

// ---------------------------------------------------------------------------------------
// Allocation-free solve (no counterpart in the paper: a deployment convenience).
//
// Some callers cannot allocate device memory at the point where they need a solve:
// frameworks whose device memory belongs to their own pool allocator, and latency-bound
// loops that forbid allocator calls (cudaMalloc / cudaFree may synchronise the device).
// ers_solve_dev_noalloc serves them: it runs the same forward/backward kernels as every
// other solve, but the kernels' scratch (the dependency counters and flags, 2 + 6 * nsn
// ints) lives in the file-scope array below instead of the context's own buffer.  The array
// is a fixed 12 MiB that every GPU loading this library keeps until the process exits;
// contexts with more than NOALLOC_MAX_SN supernodes are rejected.  All calls on a device
// share the one array, so calls whose solves overlap on the GPU race; the counters are
// cleared at each call.  The call ends with a stream synchronisation (it reads the device
// status), so it is not usable inside a stream capture.
// ---------------------------------------------------------------------------------------
namespace ers {

constexpr int NOALLOC_MAX_SN = 1 << 19;
static __device__ __align__(256) int32_t g_noalloc_sync[solve_sync_words(NOALLOC_MAX_SN)];

__global__ void k_gather_perm(int n, const int32_t* perm, const double* src, double* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}
__global__ void k_scatter_perm(int n, const int32_t* perm, const double* src, double* dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[perm[i]] = src[i];
}

// Device address of g_noalloc_sync on the current device, looked up once per device and
// kept for the life of the process (a cudaDeviceReset or a re-created primary context would
// leave the cached address stale; the library never resets a device itself).
static int32_t* noalloc_scratch(int device, cudaError_t* err) {
  static std::mutex mu;
  static int32_t* addr[128] = {};
  *err = cudaSuccess;
  if (device < 0 || device >= 128) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[device]) {
    int32_t* p = nullptr;
    *err = cudaGetSymbolAddress((void**)&p, g_noalloc_sync);
    if (*err != cudaSuccess) return nullptr;
    addr[device] = p;
  }
  return addr[device];
}

}  // namespace ers

extern "C" ers_status ers_solve_dev_noalloc(ers_ctx* c, const double* b_dev, double* x_dev) {
  using namespace ers;
  if (!c) return ERS_ERR_INVALID;
  if (c->is_group()) {
    c->err = "ers_solve_dev_noalloc: takes a context on one device";
    return ERS_ERR_INVALID;
  }
  if (!b_dev || !x_dev) {
    c->err = "ers_solve_dev_noalloc: b_dev and x_dev must not be NULL";
    return ERS_ERR_INVALID;
  }
  // both buffers must be device (or managed) memory of the context's device: a host
  // pointer or another device's memory would make the permutation kernels fault
  for (const void* ptr : {(const void*)b_dev, (const void*)x_dev}) {
    cudaPointerAttributes at{};
    cudaError_t pe = cudaPointerGetAttributes(&at, ptr);
    if (pe != cudaSuccess) {
      cudaGetLastError();   // clear the error that the failed query recorded
      c->err = std::string("ers_solve_dev_noalloc: cannot query a buffer: ") +
               cudaGetErrorString(pe);
      return ERS_ERR_INVALID;
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) ||
        at.device != c->device) {
      c->err = "ers_solve_dev_noalloc: b_dev and x_dev must be device memory of device " +
               std::to_string(c->device);
      return ERS_ERR_INVALID;
    }
  }
  if (c->plan.nsn > NOALLOC_MAX_SN) {
    c->err = "ers_solve_dev_noalloc: the factor has " + std::to_string(c->plan.nsn) +
             " supernodes, more than the allocation-free limit of " +
             std::to_string(NOALLOC_MAX_SN);
    return ERS_ERR_INVALID;
  }
  if (!c->factored) {
    c->err = "ers_solve_dev_noalloc: no factorisation of G_k yet (call ers_refactor first)";
    return ERS_ERR_INVALID;
  }
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != c->device) e = cudaSetDevice(c->device);
  int32_t* scratch = nullptr;
  if (e == cudaSuccess) scratch = noalloc_scratch(c->device, &e);
  auto cuda_fail = [&](cudaError_t err) {
    c->err = std::string("ers_solve_dev_noalloc: ") + cudaGetErrorString(err);
    if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
    return ERS_ERR_CUDA;
  };
  if (e != cudaSuccess) return cuda_fail(e);
  DevicePlan P = c->plan;
  P.sync = scratch;
  const int n = c->n;
  const int nb = (n + 255) / 256;
  e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(scratch, 0, sizeof(int32_t) * solve_sync_words(P.nsn), c->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  k_gather_perm<<<nb, 256, 0, c->stream>>>(n, c->d_perm, b_dev, c->solve_buf);
  SolveArgs A{P, c->solve_buf, n, c->d_status, c->solve_z, c->solve_part};
  launch_pair<1>(c, A, c->sm_count * c->solve_ctas_per_sm);
  k_scatter_perm<<<nb, 256, 0, c->stream>>>(n, c->d_perm, c->solve_buf, x_dev);
  c->stats.kernel_launches += 4;
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_status, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
  if (c->h_status[0] & ST_TIMEOUT) {
    c->err = "ers_solve_dev_noalloc: device wait timed out";
    return ERS_ERR_TIMEOUT;
  }
  return ERS_OK;
}
