// Arnoldi / MEVP kernels of the invert Krylov subspace method (Sec. IV, Algorithm 1).
//
//  * k_arnoldi_init : beta = ||v||, v_1 = v / beta, ||G v_1|| (scale of the Eq.-16 test)
//  * k_mgs          : modified Gram-Schmidt of w = J^-1 v_j against v_1..v_j, h_{j+1,j},
//                     v_{j+1}, happy-breakdown test, ||G v_{j+1}|| for the residual test.
//                     Cooperative launch; each thread keeps its slice of w in registers, so
//                     one pass over V_j costs 8 bytes per element; every inner product is a
//                     deterministic grid reduction (fixed block order).
//  * k_small        : exp(h H_m^-1) e_1 by scaling and squaring of the [13/13] Pade
//                     approximant in shared memory, e_m^T H_m^-1 exp(h H_m^-1) e_1, and the
//                     dimension decision of Algorithm 1 (residual of Eq. 16).
//  * k_combine      : out = a*in + sum_b c_b beta_b V_b (y_b - e_1) + sum_q d_q u_q, the
//                     ER update of Eq. 13, the error vector of Eq. 15 and ER-C (Eq. 20),
//                     optionally with max |out|.
#include "ers_internal.h"
#include "kcommon.cuh"

namespace ers {

constexpr int KB = 256;          // threads per block of the vector kernels

__constant__ double c_pade[14];  // [13/13] Pade coefficients of exp

struct CoopArgs {
  int n;
  int j;                // mgs: current column (0-based)
  int adaptive;
  VecGroup g;
  KrylovState* ks;
  const int32_t *Gp, *Gi;
  const double* Gv;
  double* part;         // partial sums: NV * gridDim
  double* out;          // reduced values
  unsigned* bar;
  unsigned* status;
};

// ||G u||^2 partial over the rows owned by this thread (row i = tid + k*T)
__device__ __forceinline__ double gnorm_part(const CoopArgs& A, const double* u, int64_t T) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += T) {
    double s = 0.0;
    for (int e = A.Gp[i]; e < A.Gp[i + 1]; ++e) s += A.Gv[e] * __ldcg(u + A.Gi[e]);
    acc += s * s;
  }
  return acc;
}

__global__ void __launch_bounds__(KB) k_arnoldi_init(CoopArgs A) {
  __shared__ double sh[KB / 32];
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nb = A.g.nb;
  double loc[MAX_RHS];
  for (int b = 0; b < MAX_RHS; ++b) loc[b] = 0.0;
  for (int b = 0; b < nb; ++b) {
    double acc = 0.0;
    for (int64_t i = tid; i < A.n; i += T) { double v = A.g.src[b][i]; acc += v * v; }
    loc[b] = block_sum(acc, sh);
  }
  grid_reduce<MAX_RHS>(loc, A.part, A.out, A.bar, A.status, sh);
  double beta[MAX_RHS];
  for (int b = 0; b < nb; ++b) beta[b] = sqrt(__ldcg(A.out + b));
  for (int b = 0; b < nb; ++b) {
    double inv = beta[b] > 0.0 ? 1.0 / beta[b] : 0.0;
    for (int64_t i = tid; i < A.n; i += T) A.g.V[b][i] = A.g.src[b][i] * inv;
  }
  double gl[MAX_RHS];
  for (int b = 0; b < MAX_RHS; ++b) gl[b] = 0.0;
  if (A.adaptive) {
    const double zero1[1] = {0.0};
    grid_reduce<1>(zero1, A.part, A.out + MAX_RHS, A.bar, A.status, sh);  // V_0 complete
    for (int b = 0; b < nb; ++b) gl[b] = block_sum(gnorm_part(A, A.g.V[b], T), sh);
    grid_reduce<MAX_RHS>(gl, A.part, A.out, A.bar, A.status, sh);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int b = 0; b < nb; ++b) {
      KrylovState& K = A.ks[A.g.slot[b]];
      K.beta = beta[b];
      K.gv1 = A.adaptive ? sqrt(__ldcg(A.out + b)) : 0.0;
      K.built = 0;
      K.m = 0;
      K.best_m = 0;
      K.best_res = INFINITY;
      K.res = INFINITY;
      K.breakdown = 0;
      K.done = beta[b] > 0.0 && isfinite(beta[b]) ? 0 : 1;
      if (!isfinite(beta[b])) atomicOr(A.status, ST_NONFINITE);
    }
  }
}

template <int EPT>
__global__ void __launch_bounds__(KB) k_mgs(CoopArgs A) {
  __shared__ double sh[KB / 32];
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nb = A.g.nb, j = A.j, n = A.n;
  const int ldh = MAX_M + 1;
  int active[MAX_RHS];
  for (int b = 0; b < nb; ++b) active[b] = !A.ks[A.g.slot[b]].done;
  double w[MAX_RHS][EPT];
  for (int b = 0; b < nb; ++b)
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      int64_t i = tid + q * T;
      w[b][q] = (active[b] && i < n) ? -A.g.src[b][i] : 0.0;
    }
  // pass 0: ||w||^2 and <w, v_0>
  double loc[2 * MAX_RHS];
  for (int b = 0; b < 2 * MAX_RHS; ++b) loc[b] = 0.0;
  for (int b = 0; b < nb; ++b) {
    double nn = 0.0, dd = 0.0;
    const double* v0 = A.g.V[b];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      int64_t i = tid + q * T;
      if (i < n) { nn += w[b][q] * w[b][q]; dd += w[b][q] * v0[i]; }
    }
    loc[2 * b] = block_sum(nn, sh);
    loc[2 * b + 1] = block_sum(dd, sh);
  }
  grid_reduce<2 * MAX_RHS>(loc, A.part, A.out, A.bar, A.status, sh);
  double w0[MAX_RHS], hcur[MAX_RHS];
  for (int b = 0; b < nb; ++b) {
    w0[b] = sqrt(__ldcg(A.out + 2 * b));
    hcur[b] = __ldcg(A.out + 2 * b + 1);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int b = 0; b < nb; ++b)
      if (active[b]) A.g.H[b][0 + j * ldh] = hcur[b];
  for (int i = 0; i <= j; ++i) {
    double lp[MAX_RHS];
    for (int b = 0; b < MAX_RHS; ++b) lp[b] = 0.0;
    for (int b = 0; b < nb; ++b) {
      const double* vi = A.g.V[b] + (int64_t)i * n;
      const double* vn = A.g.V[b] + (int64_t)(i + 1) * n;
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        int64_t e = tid + q * T;
        if (e < n) {
          w[b][q] -= hcur[b] * vi[e];
          acc += (i < j) ? w[b][q] * vn[e] : w[b][q] * w[b][q];
        }
      }
      lp[b] = block_sum(acc, sh);
    }
    grid_reduce<MAX_RHS>(lp, A.part, A.out, A.bar, A.status, sh);
    for (int b = 0; b < nb; ++b) hcur[b] = __ldcg(A.out + b);
    if (i < j && blockIdx.x == 0 && threadIdx.x == 0)
      for (int b = 0; b < nb; ++b)
        if (active[b]) A.g.H[b][(i + 1) + j * ldh] = hcur[b];
  }
  // hcur = ||w||^2 after orthogonalisation
  double hn[MAX_RHS];
  int bd[MAX_RHS];
  for (int b = 0; b < nb; ++b) {
    hn[b] = sqrt(hcur[b]);
    bd[b] = !(hn[b] > 1e-12 * w0[b]);
  }
  for (int b = 0; b < nb; ++b) {
    if (!active[b] || bd[b]) continue;
    double inv = 1.0 / hn[b];
    double* vn = A.g.V[b] + (int64_t)(j + 1) * n;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      int64_t e = tid + q * T;
      if (e < n) vn[e] = w[b][q] * inv;
    }
  }
  double gl[MAX_RHS];
  for (int b = 0; b < MAX_RHS; ++b) gl[b] = 0.0;
  if (A.adaptive) {
    const double zero1[1] = {0.0};
    grid_reduce<1>(zero1, A.part, A.out + MAX_RHS, A.bar, A.status, sh);  // v_{j+1} complete
    for (int b = 0; b < nb; ++b)
      if (active[b] && !bd[b])
        gl[b] = block_sum(gnorm_part(A, A.g.V[b] + (int64_t)(j + 1) * n, T), sh);
    grid_reduce<MAX_RHS>(gl, A.part, A.out, A.bar, A.status, sh);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int b = 0; b < nb; ++b) {
      if (!active[b]) continue;
      KrylovState& K = A.ks[A.g.slot[b]];
      A.g.H[b][(j + 1) + j * ldh] = hn[b];
      K.w0 = w0[b];
      K.built = j + 1;
      K.gvnext[j] = A.adaptive && !bd[b] ? sqrt(__ldcg(A.out + b)) : 0.0;
      if (!isfinite(hn[b])) atomicOr(A.status, ST_NONFINITE);
      if (bd[b]) { K.breakdown = 1; K.done = 1; K.m = j + 1; }
    }
  }
}

// ---------------------------------------------------------------------------------------
// small dense stage
// ---------------------------------------------------------------------------------------
__device__ void sm_matmul(double* C, const double* A, const double* B, int m) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, jj = e / m;
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc += A[i + k * m] * B[k + jj * m];
    C[e] = acc;
  }
  __syncthreads();
}

// LU with partial pivoting of M (m x m, in place); piv[k] = row swapped with k.
__device__ void sm_lu(double* M, int* piv, int m) {
  __shared__ int s_p;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(M[k + k * m]);
      for (int i = k + 1; i < m; ++i)
        if (fabs(M[i + k * m]) > best) { best = fabs(M[i + k * m]); p = i; }
      s_p = p;
      piv[k] = p;
    }
    __syncthreads();
    int p = s_p;
    if (p != k)
      for (int jj = threadIdx.x; jj < m; jj += blockDim.x) {
        double t = M[k + jj * m];
        M[k + jj * m] = M[p + jj * m];
        M[p + jj * m] = t;
      }
    __syncthreads();
    double inv = 1.0 / M[k + k * m];
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) M[i + k * m] *= inv;
    __syncthreads();
    int rem = m - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int i = k + 1 + e % rem, jj = k + 1 + e / rem;
      M[i + jj * m] -= M[i + k * m] * M[k + jj * m];
    }
    __syncthreads();
  }
}

// Solve (LU) X = B column by column in place (B: m x m); column jj by one thread.
__device__ void sm_lu_solve(const double* LU, const int* piv, double* B, int m) {
  for (int jj = threadIdx.x; jj < m; jj += blockDim.x) {
    double* b = B + jj * m;
    for (int k = 0; k < m; ++k)
      if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int i = 1; i < m; ++i) {
      double acc = b[i];
      for (int k = 0; k < i; ++k) acc -= LU[i + k * m] * b[k];
      b[i] = acc;
    }
    for (int i = m - 1; i >= 0; --i) {
      double acc = b[i];
      for (int k = i + 1; k < m; ++k) acc -= LU[i + k * m] * b[k];
      b[i] = acc / LU[i + i * m];
    }
  }
  __syncthreads();
}

// y = exp(h H^-1) e_1 for the leading m x m block of H (ld ldh); last = e_m^T H^-1 y.
// Scaling and squaring of the diagonal [13/13] Pade approximant (theta_13 = 5.37).
// Returns true when y and last are finite.  smem: 6 m^2 doubles + scratch.
__device__ bool phi_small(const double* H, int ldh, int m, double h, double* y, double* last,
                          double* smem, int* ipiv) {
  double* M0 = smem;
  double* M1 = M0 + m * m;
  double* M2 = M1 + m * m;
  double* M3 = M2 + m * m;
  double* M4 = M3 + m * m;
  double* M5 = M4 + m * m;
  double* lastrow = M5 + m * m;   // m
  double* vec = lastrow + m;      // m
  __shared__ int s_s;
  __shared__ double s_norm;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, jj = e / m;
    M0[e] = H[i + jj * ldh];
    M1[e] = (i == jj) ? h : 0.0;
  }
  __syncthreads();
  sm_lu(M0, ipiv, m);
  sm_lu_solve(M0, ipiv, M1, m);          // M1 = X = h H^-1
  for (int k = threadIdx.x; k < m; k += blockDim.x) lastrow[k] = M1[(m - 1) + k * m] / h;
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int jj = 0; jj < m; ++jj) {
      double cs = 0.0;
      for (int i = 0; i < m; ++i) cs += fabs(M1[i + jj * m]);
      nrm = fmax(nrm, cs);
    }
    s_norm = nrm;
    int s = 0;
    if (nrm > 5.371920351148152) s = (int)ceil(log2(nrm / 5.371920351148152));
    if (!isfinite(nrm)) s = 0;
    s_s = min(s, 1000);
  }
  __syncthreads();
  int s = s_s;
  if (!isfinite(s_norm)) {
    if (threadIdx.x == 0) *last = NAN;
    for (int k = threadIdx.x; k < m; k += blockDim.x) y[k] = NAN;
    __syncthreads();
    return false;
  }
  double sc = ldexp(1.0, -s);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) M1[e] *= sc;
  __syncthreads();
  sm_matmul(M2, M1, M1, m);   // A2
  sm_matmul(M3, M2, M2, m);   // A4
  sm_matmul(M4, M3, M2, m);   // A6
  for (int e = threadIdx.x; e < m * m; e += blockDim.x)
    M0[e] = c_pade[13] * M4[e] + c_pade[11] * M3[e] + c_pade[9] * M2[e];
  __syncthreads();
  sm_matmul(M5, M4, M0, m);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, jj = e / m;
    M5[e] += c_pade[7] * M4[e] + c_pade[5] * M3[e] + c_pade[3] * M2[e] + (i == jj ? c_pade[1] : 0.0);
  }
  __syncthreads();
  sm_matmul(M0, M1, M5, m);   // U
  for (int e = threadIdx.x; e < m * m; e += blockDim.x)
    M5[e] = c_pade[12] * M4[e] + c_pade[10] * M3[e] + c_pade[8] * M2[e];
  __syncthreads();
  sm_matmul(M1, M4, M5, m);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, jj = e / m;
    double V = M1[e] + c_pade[6] * M4[e] + c_pade[4] * M3[e] + c_pade[2] * M2[e] +
               (i == jj ? c_pade[0] : 0.0);
    M2[e] = V - M0[e];
    M3[e] = V + M0[e];
  }
  __syncthreads();
  sm_lu(M2, ipiv, m);
  sm_lu_solve(M2, ipiv, M3, m);   // R = (V - U)^-1 (V + U)
  double* R = M3;
  double* Tm = M4;
  for (int q = 0; q + 1 < s; ++q) {
    sm_matmul(Tm, R, R, m);
    double* t = R; R = Tm; Tm = t;
  }
  // y = R (R e_1) when s >= 1, else R e_1
  for (int i = threadIdx.x; i < m; i += blockDim.x) vec[i] = R[i];
  __syncthreads();
  if (s >= 1) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double acc = 0.0;
      for (int k = 0; k < m; ++k) acc += R[i + k * m] * vec[k];
      y[i] = acc;
    }
  } else {
    for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = vec[i];
  }
  __syncthreads();
  __shared__ int s_fin;
  if (threadIdx.x == 0) {
    double acc = 0.0;
    bool fin = true;
    for (int k = 0; k < m; ++k) {
      acc += lastrow[k] * y[k];
      fin = fin && isfinite(y[k]);
    }
    *last = acc;
    s_fin = fin && isfinite(acc);
  }
  __syncthreads();
  return s_fin;
}


struct SmallArgs {
  int mode;
  int nb;
  int slot[MAX_RHS];
  const double* H[MAX_RHS];
  KrylovState* ks;
  double h, eps;
  int m_min, m_max;
  unsigned* status;
  // test mode
  const double* Htest; int ldh_test; int m_test; double* y_out; double* last_out;
};

__global__ void k_small(SmallArgs A) {
  extern __shared__ double smem[];
  __shared__ int ipiv[MAX_M];
  __shared__ double ybuf[MAX_M];
  __shared__ double s_last;
  const int ldh = MAX_M + 1;
  if (A.mode == SMALL_TEST) {
    bool fin = phi_small(A.Htest, A.ldh_test, A.m_test, A.h, ybuf, &s_last, smem, ipiv);
    (void)fin;
    for (int k = threadIdx.x; k < A.m_test; k += blockDim.x) A.y_out[k] = ybuf[k];
    if (threadIdx.x == 0) *A.last_out = s_last;
    return;
  }
  int b = blockIdx.x;
  KrylovState& K = A.ks[A.slot[b]];
  const double* H = A.H[b];
  __shared__ int s_done, s_m, s_built, s_bd, s_m_in;
  if (threadIdx.x == 0) {
    s_done = K.done; s_m = K.m; s_built = K.built; s_bd = K.breakdown;
    s_m_in = (K.beta > 0.0);
  }
  __syncthreads();
  if (!s_m_in) return;   // zero vector: MEVP = 0
  auto write_y = [&](int m) {
    for (int k = threadIdx.x; k < m; k += blockDim.x) K.y[k] = ybuf[k];
    if (threadIdx.x == 0) { K.last = s_last; K.m = m; }
  };
  // dimension at a breakdown: built, or built-1 when the last direction was noise
  auto finalize_breakdown = [&]() {
    int m = s_built;
    bool fin = phi_small(H, ldh, m, A.h, ybuf, &s_last, smem, ipiv);
    if (!fin && m > 1) {
      m -= 1;
      fin = phi_small(H, ldh, m, A.h, ybuf, &s_last, smem, ipiv);
    }
    if (!fin && threadIdx.x == 0) atomicOr(A.status, ST_KRYLOV);
    write_y(m);
  };
  if (A.mode == SMALL_FINAL) {
    bool fin = phi_small(H, ldh, s_m, A.h, ybuf, &s_last, smem, ipiv);
    if (!fin && threadIdx.x == 0) atomicOr(A.status, ST_KRYLOV);
    write_y(s_m);
    return;
  }
  if (A.mode == SMALL_FIXED_END) {
    if (s_bd) { finalize_breakdown(); return; }
    bool fin = phi_small(H, ldh, s_built, A.h, ybuf, &s_last, smem, ipiv);
    if (!fin && threadIdx.x == 0) atomicOr(A.status, ST_KRYLOV);
    write_y(s_built);
    if (threadIdx.x == 0) K.done = 1;
    return;
  }
  // SMALL_RESID: called after every Arnoldi iteration in adaptive mode
  if (s_done && !s_bd) return;   // already converged earlier
  if (s_bd) {
    if (s_m == s_built) { finalize_breakdown(); if (threadIdx.x == 0) K.breakdown = 2; }
    return;
  }
  int jj = s_built;
  if (jj >= A.m_min) {
    bool fin = phi_small(H, ldh, jj, A.h, ybuf, &s_last, smem, ipiv);
    __shared__ int s_conv;
    if (threadIdx.x == 0) {
      double res = H[jj + (jj - 1) * ldh] * K.gvnext[jj - 1] * fabs(s_last) / K.gv1;
      if (!fin) res = INFINITY;
      K.res = res;
      if (isfinite(res) && res < K.best_res) { K.best_res = res; K.best_m = jj; }
      s_conv = isfinite(res) && res < A.eps;
    }
    __syncthreads();
    if (s_conv) {
      write_y(jj);
      if (threadIdx.x == 0) K.done = 1;
      return;
    }
  }
  if (jj >= A.m_max) {
    // never converged: the dimension with the smallest finite residual
    int m = K.best_m > 0 ? K.best_m : jj;
    __syncthreads();
    bool fin = phi_small(H, ldh, m, A.h, ybuf, &s_last, smem, ipiv);
    if (!fin && threadIdx.x == 0) atomicOr(A.status, ST_KRYLOV);
    write_y(m);
    if (threadIdx.x == 0) K.done = 1;
  }
}

// out = a*in + sum_b c_b beta_b V_b (y_b - e_1) + d0 u0 + d1 u1; optional max|out| into
// maxout (as ordered bits of a non-negative double).
struct CombineArgs {
  int n;
  double* out;
  const double* in; double a;
  int nb;
  const double* V[MAX_RHS]; int slot[MAX_RHS]; double c[MAX_RHS];
  const KrylovState* ks;
  const double* u0; double d0;
  const double* u1; double d1;
  unsigned long long* maxout;
};

__global__ void __launch_bounds__(KB) k_combine(CombineArgs A) {
  __shared__ double ys[MAX_RHS][MAX_M];
  __shared__ double coef[MAX_RHS];
  __shared__ int ms[MAX_RHS];
  __shared__ double sh[KB / 32];
  for (int b = 0; b < A.nb; ++b) {
    const KrylovState& K = A.ks[A.slot[b]];
    if (threadIdx.x == 0) {
      ms[b] = K.beta > 0.0 ? K.m : 0;
      coef[b] = A.c[b] * K.beta;
    }
    for (int k = threadIdx.x; k < MAX_M; k += blockDim.x) ys[b][k] = K.y[k];
  }
  __syncthreads();
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = A.in ? A.a * A.in[i] : 0.0;
    for (int b = 0; b < A.nb; ++b) {
      int m = ms[b];
      if (m == 0) continue;
      const double* Vb = A.V[b];
      double acc = (ys[b][0] - 1.0) * Vb[i];
      for (int k = 1; k < m; ++k) acc += ys[b][k] * Vb[(int64_t)k * A.n + i];
      v += coef[b] * acc;
    }
    if (A.u0) v += A.d0 * A.u0[i];
    if (A.u1) v += A.d1 * A.u1[i];
    A.out[i] = v;
    mx = fmax(mx, fabs(v));
    if (!isfinite(v)) mx = INFINITY;
  }
  if (A.maxout) {
    mx = block_max(mx, sh);
    if (threadIdx.x == 0) atomicMax(A.maxout, (unsigned long long)__double_as_longlong(mx));
  }
}

// max |x| over n (non-negative bits compare as integers)
__global__ void __launch_bounds__(KB) k_absmax(int n, const double* x, unsigned long long* out) {
  __shared__ double sh[KB / 32];
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = fabs(x[i]);
    mx = isfinite(v) ? fmax(mx, v) : INFINITY;
  }
  mx = block_max(mx, sh);
  if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
cudaError_t krylov_init_constants() {
  // [q/q] Pade approximant of exp: c_k = (2q-k)! q! / ((2q)! k! (q-k)!), q = 13
  double c[14];
  const int q = 13;
  for (int k = 0; k <= q; ++k) {
    double v = 1.0;
    for (int i = 1; i <= q; ++i) v *= (double)i;            // q!
    for (int i = 1; i <= 2 * q - k; ++i) v *= (double)i;    // (2q-k)!
    for (int i = 1; i <= 2 * q; ++i) v /= (double)i;        // (2q)!
    for (int i = 1; i <= k; ++i) v /= (double)i;            // k!
    for (int i = 1; i <= q - k; ++i) v /= (double)i;        // (q-k)!
    c[k] = v;
  }
  cudaError_t e = cudaMemcpyToSymbol(c_pade, c, sizeof(c));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (6 * MAX_M * MAX_M + 2 * MAX_M) * 8);
}

static int coop_blocks_for(ers_ctx* c, int n) {
  int want = (n + KB - 1) / KB;
  return std::max(1, std::min(want, c->coop_blocks));
}

static CoopArgs make_coop(ers_ctx* c, const VecGroup& g, int j, int adaptive) {
  CoopArgs A;
  A.n = c->n;
  A.j = j;
  A.adaptive = adaptive;
  A.g = g;
  A.ks = c->ks;
  A.Gp = c->G_ptr;
  A.Gi = c->G_idx;
  A.Gv = c->G_val;
  A.part = c->red;
  A.out = c->red + 2 * MAX_RHS * 4096;
  A.bar = c->d_status + 4;
  A.status = c->d_status;
  return A;
}

cudaError_t launch_arnoldi_init(ers_ctx* c, const VecGroup& g, int adaptive) {
  CoopArgs A = make_coop(c, g, 0, adaptive);
  int blocks = coop_blocks_for(c, c->n);
  void* args[] = {&A};
  c->stats.kernel_launches++;
  return cudaLaunchCooperativeKernel((void*)k_arnoldi_init, blocks, KB, args, 0, c->stream);
}

cudaError_t launch_mgs(ers_ctx* c, const VecGroup& g, int j, int adaptive) {
  CoopArgs A = make_coop(c, g, j, adaptive);
  int blocks = coop_blocks_for(c, c->n);
  int64_t T = (int64_t)blocks * KB;
  int ept = (int)((c->n + T - 1) / T);
  void* args[] = {&A};
  c->stats.kernel_launches++;
  if (ept <= 1) return cudaLaunchCooperativeKernel((void*)k_mgs<1>, blocks, KB, args, 0, c->stream);
  if (ept <= 2) return cudaLaunchCooperativeKernel((void*)k_mgs<2>, blocks, KB, args, 0, c->stream);
  if (ept <= 4) return cudaLaunchCooperativeKernel((void*)k_mgs<4>, blocks, KB, args, 0, c->stream);
  if (ept <= 8) return cudaLaunchCooperativeKernel((void*)k_mgs<8>, blocks, KB, args, 0, c->stream);
  if (ept <= 16) return cudaLaunchCooperativeKernel((void*)k_mgs<16>, blocks, KB, args, 0, c->stream);
  return cudaErrorInvalidValue;
}

cudaError_t launch_small(ers_ctx* c, int mode, const VecGroup& g, double h, int m_max) {
  SmallArgs A{};
  A.mode = mode;
  A.nb = g.nb;
  for (int b = 0; b < g.nb; ++b) { A.slot[b] = g.slot[b]; A.H[b] = g.H[b]; }
  A.ks = c->ks;
  A.h = h;
  A.eps = c->opts.eps_krylov;
  A.m_min = c->opts.m_min;
  A.m_max = m_max;
  A.status = c->d_status;
  size_t sm = (6 * (size_t)MAX_M * MAX_M + 2 * MAX_M) * 8;
  k_small<<<g.nb, KB, sm, c->stream>>>(A);
  c->stats.kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_small_test(ers_ctx* c, const double* H, int ldh, int m, double h, double* y,
                              double* last) {
  SmallArgs A{};
  A.mode = SMALL_TEST;
  A.h = h;
  A.Htest = H;
  A.ldh_test = ldh;
  A.m_test = m;
  A.y_out = y;
  A.last_out = last;
  size_t sm = (6 * (size_t)m * m + 2 * (size_t)m) * 8;
  k_small<<<1, KB, sm, c->stream>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_combine(ers_ctx* c, double* out, const double* in, double a, const VecGroup* g,
                           const double* cb, const double* u0, double d0, const double* u1,
                           double d1, unsigned long long* maxout) {
  CombineArgs A{};
  A.n = c->n;
  A.out = out;
  A.in = in;
  A.a = a;
  A.nb = g ? g->nb : 0;
  for (int b = 0; b < A.nb; ++b) { A.V[b] = g->V[b]; A.slot[b] = g->slot[b]; A.c[b] = cb[b]; }
  A.ks = c->ks;
  A.u0 = u0; A.d0 = d0; A.u1 = u1; A.d1 = d1;
  A.maxout = maxout;
  int blocks = std::min(c->sm_count * 8, (c->n + KB - 1) / KB);
  k_combine<<<std::max(blocks, 1), KB, 0, c->stream>>>(A);
  c->stats.kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_absmax(ers_ctx* c, const double* x, unsigned long long* out) {
  int blocks = std::min(c->sm_count * 8, (c->n + KB - 1) / KB);
  k_absmax<<<std::max(blocks, 1), KB, 0, c->stream>>>(c->n, x, out);
  c->stats.kernel_launches++;
  return cudaGetLastError();
}

int coop_max_blocks(int sm_count) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mgs<16>, KB, 0);
  int per_sm2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, k_arnoldi_init, KB, 0);
  per_sm = std::min(per_sm, per_sm2);
  return std::max(1, std::min(per_sm, 4) * sm_count);
}

}  // namespace ers
