// Sparse matrix-vector products and the supernodal triangular solves with the factors
// of G_k (Algorithm 1: "Solve -G w = C v_j"; Alg. 2's setup solves).
//
// The solves are persistent, warp-granular and sync-free: every warp takes the next task
// of a topologically ordered list (atomic counter), waits on a dependency word (bounded
// spin), runs the task with its 32 lanes and publishes completion.  Because tasks are
// taken in list order and only wait on earlier tasks, the scheme cannot deadlock.
//   forward  (L y = b):  FUSED/DIAG wait until every unit scattering into the supernode is
//                        done; y_s <- L11^-1 y_s; OFF/FUSED scatter y_R -= L21 y_s (FP64
//                        atomics) and bump the counters of the supernodes they touched.
//   backward (U x = y):  a supernode's rows R_off lie in its ancestors, and a parent is
//                        finished only after its own parent, so waiting for the parent
//                        suffices; x_s <- U11^-1 (x_s - U12 x_R).
// Up to MAX_RHS right-hand sides (stride n) share each pass over the factors.
#include "ers_internal.h"
#include "kcommon.cuh"

namespace ers {

constexpr int SOLVE_WARPS = 8;   // warps per block

// y = A x for a CSR matrix (warp per row for long rows is not needed: rows here are short)
__global__ void k_spmv(int nrows, const int32_t* ptr, const int32_t* idx, const double* val,
                       const double* x, double* y, double alpha) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  double acc = 0.0;
  for (int e = ptr[i]; e < ptr[i + 1]; ++e) acc += val[e] * x[idx[e]];
  y[i] = alpha * acc;
}

// y_r = alpha * C v_r for several vectors (used to form the Arnoldi right-hand sides)
__global__ void k_spmv_multi(int n, const int32_t* ptr, const int32_t* idx, const double* val,
                             const double* const* xs, double* y, int64_t ystride, int nv,
                             double alpha) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int v = 0; v < nv; ++v) {
    const double* x = xs[v];
    double acc = 0.0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) acc += val[e] * x[idx[e]];
    y[v * ystride + i] = alpha * acc;
  }
}

struct SolveArgs {
  DevicePlan P;
  double* y;        // nrhs vectors, stride n (in place)
  int nrhs;
  int n;
  unsigned* status;
};

// sync words layout (ints): [0] fwd task counter, [1] bwd task counter,
// [2 + s] fwd arrivals, [2 + nsn + s] ready/done flags, [2 + 2 nsn + s] bwd arrivals
__global__ void __launch_bounds__(32 * SOLVE_WARPS) k_trsv_fwd(SolveArgs A) {
  __shared__ double ys[SOLVE_WARPS][MAX_RHS][64];
  const DevicePlan& P = A.P;
  int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  int32_t* sync = P.sync;
  int32_t* arrive = sync + 2;
  int32_t* ready = sync + 2 + P.nsn;
  const int n = A.n, nrhs = A.nrhs;
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(sync, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= P.nfwd) break;
    SolveTask T = P.fwd[t];
    int s = T.sn;
    int c0 = P.sn_start[s], w = P.sn_start[s + 1] - c0;
    int r = (int)(P.rptr[s + 1] - P.rptr[s]);
    int ok = 1;
    if (lane == 0) {
      if (T.kind == TASK_OFF) ok = wait_geq(ready + s, 1, A.status);
      else ok = wait_geq(arrive + s, P.fwd_expect[s], A.status);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) continue;
    __threadfence();
    // load y_s
    for (int q = lane; q < w; q += 32)
      for (int k = 0; k < nrhs; ++k) ys[wq][k][q] = __ldcg(A.y + (int64_t)k * n + c0 + q);
    __syncwarp();
    if (T.kind != TASK_OFF) {
      // z = L11^-1 y_s (unit lower, column-major w x w)
      const double* Li = P.LDi + P.d_off[s];
      double z[2][MAX_RHS];
      for (int h = 0; h < 2; ++h) {
        int q = lane + 32 * h;
        for (int k = 0; k < nrhs; ++k) z[h][k] = 0.0;
        if (q < w)
          for (int j = 0; j <= q; ++j) {
            double l = Li[q + j * w];
            for (int k = 0; k < nrhs; ++k) z[h][k] += l * ys[wq][k][j];
          }
      }
      __syncwarp();
      for (int h = 0; h < 2; ++h) {
        int q = lane + 32 * h;
        if (q < w)
          for (int k = 0; k < nrhs; ++k) {
            ys[wq][k][q] = z[h][k];
            A.y[(int64_t)k * n + c0 + q] = z[h][k];
          }
      }
      __syncwarp();
    }
    if (T.kind == TASK_DIAG) {
      if (lane == 0) {
        __threadfence();
        st_release(ready + s, 1);
      }
      continue;
    }
    // scatter rows r0..r1: y[R[i]] -= sum_k Lo[i + k r] z_k
    const double* Lo = P.Lo + P.o_off[s];
    const int32_t* R = P.rows + P.rptr[s];
    for (int i = T.r0 + lane; i < T.r1; i += 32) {
      double acc[MAX_RHS];
      for (int k = 0; k < nrhs; ++k) acc[k] = 0.0;
      for (int j = 0; j < w; ++j) {
        double l = __ldg(Lo + i + (int64_t)j * r);
        for (int k = 0; k < nrhs; ++k) acc[k] += l * ys[wq][k][j];
      }
      int row = R[i];
      for (int k = 0; k < nrhs; ++k) atomicAdd(A.y + (int64_t)k * n + row, -acc[k]);
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      for (int q = 0; q < T.ntgt; ++q) red_release_add(arrive + P.fwd_tgt[T.tgt0 + q], 1);
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(32 * SOLVE_WARPS) k_trsv_bwd(SolveArgs A) {
  __shared__ double xs[SOLVE_WARPS][MAX_RHS][64];
  const DevicePlan& P = A.P;
  int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  int32_t* sync = P.sync;
  int32_t* done = sync + 2 + P.nsn;
  int32_t* arriveb = sync + 2 + 2 * P.nsn;
  const int n = A.n, nrhs = A.nrhs;
  while (true) {
    int t = 0;
    if (lane == 0) t = atomicAdd(sync + 1, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= P.nbwd) break;
    SolveTask T = P.bwd[t];
    int s = T.sn;
    int c0 = P.sn_start[s], w = P.sn_start[s + 1] - c0;
    int r = (int)(P.rptr[s + 1] - P.rptr[s]);
    int p = P.sn_parent[s];
    int ok = 1;
    if (lane == 0) {
      if (T.kind == TASK_DIAG) ok = wait_geq(arriveb + s, P.bwd_nchunk[s], A.status);
      else if (p >= 0) ok = wait_geq(done + p, 2, A.status);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) continue;
    __threadfence();
    if (T.kind != TASK_DIAG) {
      // partial z_k = sum_{i in r0..r1} Uo[i + k r] x[R[i]]
      const double* Uo = P.Uo + P.o_off[s];
      const int32_t* R = P.rows + P.rptr[s];
      double xr[8][MAX_RHS];
      int nchunk = (T.r1 - T.r0 + 31) / 32;
      // rows are processed 32 at a time; gather x[R[i]] once per row block
      for (int k = 0; k < nrhs; ++k)
        for (int q = lane; q < w; q += 32) xs[wq][k][q] = 0.0;
      __syncwarp();
      for (int cb = 0; cb < nchunk; cb += 8) {
        int nb = min(8, nchunk - cb);
        for (int b = 0; b < nb; ++b) {
          int i = T.r0 + (cb + b) * 32 + lane;
          for (int k = 0; k < nrhs; ++k)
            xr[b][k] = i < T.r1 ? __ldcg(A.y + (int64_t)k * n + R[i]) : 0.0;
        }
        for (int j = 0; j < w; ++j) {
          double acc[MAX_RHS];
          for (int k = 0; k < nrhs; ++k) acc[k] = 0.0;
          for (int b = 0; b < nb; ++b) {
            int i = T.r0 + (cb + b) * 32 + lane;
            double u = i < T.r1 ? __ldg(Uo + i + (int64_t)j * r) : 0.0;
            for (int k = 0; k < nrhs; ++k) acc[k] += u * xr[b][k];
          }
          for (int k = 0; k < nrhs; ++k) {
            double v = warp_sum(acc[k]);
            if (lane == 0) xs[wq][k][j] += v;
          }
        }
      }
      __syncwarp();
      if (T.kind == TASK_OFF) {
        for (int q = lane; q < w; q += 32)
          for (int k = 0; k < nrhs; ++k) atomicAdd(A.y + (int64_t)k * n + c0 + q, -xs[wq][k][q]);
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          red_release_add(arriveb + s, 1);
        }
        __syncwarp();
        continue;
      }
      // FUSED: x_s = y_s - z
      for (int q = lane; q < w; q += 32)
        for (int k = 0; k < nrhs; ++k)
          xs[wq][k][q] = __ldcg(A.y + (int64_t)k * n + c0 + q) - xs[wq][k][q];
    } else {
      for (int q = lane; q < w; q += 32)
        for (int k = 0; k < nrhs; ++k) xs[wq][k][q] = __ldcg(A.y + (int64_t)k * n + c0 + q);
    }
    __syncwarp();
    // x_s <- U11^-1 x_s (upper, column-major)
    const double* Ui = P.UDi + P.d_off[s];
    double z[2][MAX_RHS];
    for (int h = 0; h < 2; ++h) {
      int q = lane + 32 * h;
      for (int k = 0; k < nrhs; ++k) z[h][k] = 0.0;
      if (q < w)
        for (int j = q; j < w; ++j) {
          double u = Ui[q + j * w];
          for (int k = 0; k < nrhs; ++k) z[h][k] += u * xs[wq][k][j];
        }
    }
    for (int h = 0; h < 2; ++h) {
      int q = lane + 32 * h;
      if (q < w)
        for (int k = 0; k < nrhs; ++k) A.y[(int64_t)k * n + c0 + q] = z[h][k];
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      st_release(done + s, 2);
    }
    __syncwarp();
  }
}

void launch_spmv(ers_ctx* c, const int32_t* ptr, const int32_t* idx, const double* val,
                 const double* x, double* y, double alpha) {
  k_spmv<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->n, ptr, idx, val, x, y, alpha);
  c->stats.kernel_launches++;
}

// Solve G_k X = Y in place for nrhs vectors (stride n) of c->solve_buf or any buffer.
cudaError_t launch_solve(ers_ctx* c, double* y, int nrhs) {
  DevicePlan& P = c->plan;
  cudaError_t e = cudaMemsetAsync(P.sync, 0, sizeof(int32_t) * (2 + 3 * (size_t)P.nsn), c->stream);
  if (e != cudaSuccess) return e;
  SolveArgs A{P, y, nrhs, c->n, c->d_status};
  int blocks = c->sm_count * 8;
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
  k_trsv_fwd<<<blocks, 32 * SOLVE_WARPS, 0, c->stream>>>(A);
  k_trsv_bwd<<<blocks, 32 * SOLVE_WARPS, 0, c->stream>>>(A);
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

}  // namespace ers
