// Small dense stage of the invert-Krylov MEVP (Sec. IV, Eq. 14 and Eq. 16), shared by the
// single-circuit and the batched kernels: exp(h H_m^-1) e_1 by scaling and squaring of the
// diagonal [13/13] Pade approximant in shared memory, e_m^T H_m^-1 exp(h H_m^-1) e_1, and the
// Krylov-dimension decision of Algorithm 1.
#pragma once
#include "ers_internal.h"

namespace ers {

// Constants of the small dense stage: the [13/13] Pade coefficients, and whether the
// near-null eigenvalues of H_m are deflated first (a C with capacitor-free nodes).
struct PadeCoef {
  double c[14];
  int deflate = 0;
};

// shared memory (doubles) of the small dense stage for dimension m
constexpr size_t small_smem_doubles(size_t m) { return 6 * m * m + 10 * m; }

// [q/q] Pade approximant of exp: c_k = (2q-k)! q! / ((2q)! k! (q-k)!), q = 13
inline PadeCoef pade_coefficients(int deflate = 0) {
  PadeCoef P;
  P.deflate = deflate;
  const int q = 13;
  for (int k = 0; k <= q; ++k) {
    double v = 1.0;
    for (int i = 1; i <= q; ++i) v *= (double)i;            // q!
    for (int i = 1; i <= 2 * q - k; ++i) v *= (double)i;    // (2q-k)!
    for (int i = 1; i <= 2 * q; ++i) v /= (double)i;        // (2q)!
    for (int i = 1; i <= k; ++i) v /= (double)i;            // k!
    for (int i = 1; i <= q - k; ++i) v /= (double)i;        // (q-k)!
    P.c[k] = v;
  }
  return P;
}

// ---- a cluster of CS CTAs on one small dense problem ------------------------------------
// GB300 issues FP64 at 2 FMA/clk/SM, so the m^3 products of the scaling and squaring take
// tens of microseconds on one SM.  With CS > 1 each CTA of a thread-block cluster computes a
// slab of columns of every product (and of the two multi-column LU solves) and stores it
// into every CTA's copy through distributed shared memory; everything else (the LU
// factorisations, the elementwise steps, the decisions) runs redundantly in every CTA on
// identical data, so all CTAs hold the same bits and take the same branches.  Each element is
// computed with the same operations in the same order as with CS = 1: the results are the
// single-CTA results bit for bit.
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; orders the distributed stores before it
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_store(double* p, unsigned rank, double v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}
// the columns [j0, j1) of an m-column result this CTA computes
template <int CS>
__device__ __forceinline__ void cl_slab(int m, int& j0, int& j1) {
  if constexpr (CS == 1) {
    j0 = 0;
    j1 = m;
  } else {
    const int w = (m + CS - 1) / CS;
    j0 = min(m, (int)cl_rank() * w);
    j1 = min(m, j0 + w);
  }
}

// Small dense products and solves run across the cluster from this dimension on; below it
// every CTA computes them whole (the exchange would cost more than the FMAs it splits).
constexpr int CL_MIN_M = 20;

// C = A B (m x m, column-major).  CS > 1 and m >= CL_MIN_M: C's slab goes to every CTA; no
// CTA may read C between the previous cluster barrier and this call (phi_small keeps that).
template <int CS = 1>
__device__ inline void sm_matmul(double* C, const double* A, const double* B, int m) {
  const bool split = CS > 1 && m >= CL_MIN_M;
  int j0 = 0, j1 = m;
  if (split) cl_slab<CS>(m, j0, j1);
  const int ne = (j1 - j0) * m;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const int i = e % m, jj = j0 + e / m;
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc += A[i + k * m] * B[k + jj * m];
    C[i + jj * m] = acc;
    if constexpr (CS > 1) {
      if (split) {
        const unsigned r = cl_rank();
        for (int q = 1; q < CS; ++q) cl_store(C + i + jj * m, (r + q) % CS, acc);
      }
    }
  }
  if (split) {
    if constexpr (CS > 1) cl_sync();
  } else {
    __syncthreads();
  }
}

// LU with partial pivoting of M (m x m, column-major, in place); piv[k] = row swapped with k;
// rdiag (m doubles, may be nullptr) receives 1 / U[k,k].
// GB300 runs FP64 at 2 FMA/clk/SM, so every FP64 instruction of a warp costs tens of
// cycles; the per-column critical path is kept short: warp 0 finds the pivot comparing the
// bit patterns of |M[i,k]| as integers (same order as the values for finite entries; ties to
// the lowest row) and its lane 0 forms the one reciprocal inv = 1 / pivot; then the CTA swaps
// rows k and p and forms the multipliers l_i = M[i,k] * inv; then the trailing update
// M[i,j] -= l_i M[k,j] and column k = l.  Three barriers per column.  floor > 0: a pivot
// below it is raised to it (sign kept).
__device__ inline void sm_lu(double* M, int* piv, int m, double floor = 0.0,
                             double* rdiag = nullptr) {
  __shared__ int s_p;
  __shared__ double s_inv, s_pv;
  __shared__ double s_l[MAX_M];
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < m; ++k) {
    if (threadIdx.x < 32) {
      unsigned long long best = 0ull;
      int p = 0x7fffffff;                      // a lane without rows loses every tie
      for (int i = k + lane; i < m; i += 32) {
        const unsigned long long v =
            (unsigned long long)__double_as_longlong(M[i + k * m]) & 0x7fffffffffffffffull;
        if (p == 0x7fffffff || v > best) { best = v; p = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > best || (ob == best && op < p)) { best = ob; p = op; }
      }
      if (lane == 0) {
        s_p = p;
        piv[k] = p;
        double v = M[p + k * m];
        if (floor > 0.0 && fabs(v) < floor) v = v < 0.0 ? -floor : floor;
        s_pv = v;
        s_inv = 1.0 / v;
        if (rdiag) rdiag[k] = s_inv;
      }
    }
    __syncthreads();
    const int p = s_p;
    const double inv = s_inv;
    // rows k and p swap in every column but k; column k below the diagonal becomes the
    // multipliers (its row p holds the old M[k,k] after the swap)
    if (p != k)
      for (int jj = threadIdx.x; jj < m; jj += blockDim.x)
        if (jj != k) {
          double t = M[k + jj * m];
          M[k + jj * m] = M[p + jj * m];
          M[p + jj * m] = t;
        }
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x)
      s_l[i] = (i == p ? M[k + k * m] : M[i + k * m]) * inv;
    __syncthreads();
    if (threadIdx.x == 0) M[k + k * m] = s_pv;
    const int rem = m - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int i = k + 1 + e % rem, jj = k + 1 + e / rem;
      M[i + jj * m] -= s_l[i] * M[k + jj * m];
    }
    for (int i = k + 1 + threadIdx.x; i < m; i += blockDim.x) M[i + k * m] = s_l[i];
    __syncthreads();
  }
}

// Solve (LU) X = B in place (B: m x m, column-major) with rdiag = 1 / U[k,k] from sm_lu: the
// row permutation, then forward and backward substitution row by row, each step's update
// spread over the CTA's threads one element each (lane-dense: on GB300 an FP64 warp
// instruction costs the same with idle lanes).  Backward step k scales row k by rdiag[k] and
// updates the rows above with the scaled value, which every thread forms itself; the scaled
// row k is stored one step later, when no thread reads it any more: one barrier per step.
//
// CS > 1 and m >= CL_MIN_M: each CTA solves its slab of B's columns and sends it to every
// other CTA; a cluster barrier first makes sure that no CTA still writes B locally.
template <int CS = 1>
__device__ inline void sm_lu_solve(const double* LU, const int* piv, const double* rdiag,
                                   double* B, int m) {
  const bool split = CS > 1 && m >= CL_MIN_M;
  int j0 = 0, j1 = m;
  if (split) cl_slab<CS>(m, j0, j1);
  const int nc = j1 - j0;
  if constexpr (CS > 1) {
    if (split) cl_sync();
  }
  for (int jj = j0 + threadIdx.x; jj < j1; jj += blockDim.x) {
    double* b = B + (size_t)jj * m;
    for (int k = 0; k < m; ++k)
      if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
  }
  __syncthreads();
  for (int k = 0; k < m - 1; ++k) {          // L (unit diagonal): B[i,:] -= L[i,k] B[k,:]
    const int rem = m - k - 1;
    for (int e = threadIdx.x; e < rem * nc; e += blockDim.x) {
      int i = k + 1 + e % rem, jj = j0 + e / rem;
      B[i + jj * m] -= LU[i + k * m] * B[k + jj * m];
    }
    __syncthreads();
  }
  for (int k = m - 1; k >= 0; --k) {         // U: x_k = B[k,:] rdiag[k]; B[i,:] -= U[i,k] x_k
    const double rd = rdiag[k];
    for (int e = threadIdx.x; e < k * nc; e += blockDim.x) {
      int i = e % k, jj = j0 + e / k;
      B[i + jj * m] -= LU[i + k * m] * (B[k + jj * m] * rd);
    }
    if (k + 1 < m)                           // row k + 1 is final now: store it scaled
      for (int jj = j0 + threadIdx.x; jj < j1; jj += blockDim.x)
        B[k + 1 + jj * m] *= rdiag[k + 1];
    __syncthreads();
  }
  for (int jj = j0 + threadIdx.x; jj < j1; jj += blockDim.x) B[jj * m] *= rdiag[0];
  __syncthreads();
  if constexpr (CS > 1) {
    if (split) {
      const unsigned r = cl_rank();
      const int ne = nc * m;
      for (int e = threadIdx.x; e < ne * (CS - 1); e += blockDim.x) {
        const int q = 1 + e / ne, el = e % ne;
        double* pe = B + (size_t)j0 * m + el;
        cl_store(pe, (r + q) % CS, *pe);
      }
      cl_sync();
    }
  }
}

// x <- A^-1 x (trans = false) or A^-T x (trans = true) with the LU of sm_lu (P A = L U, L
// unit lower; A^T = U^T L^T P).  Run by one warp; the caller synchronises around it.
__device__ inline void warp_lu_solve_vec(const double* LU, const int* piv, double* x, int m,
                                         bool trans) {
  const int lane = threadIdx.x & 31;
  if (!trans) {
    if (lane == 0)
      for (int k = 0; k < m; ++k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    __syncwarp();
    for (int k = 0; k < m; ++k) {              // L y = P x
      const double xk = x[k];
      for (int i = k + 1 + lane; i < m; i += 32) x[i] -= LU[i + k * m] * xk;
      __syncwarp();
    }
    for (int k = m - 1; k >= 0; --k) {         // U z = y
      if (lane == 0) x[k] /= LU[k + k * m];
      __syncwarp();
      const double xk = x[k];
      for (int i = lane; i < k; i += 32) x[i] -= LU[i + k * m] * xk;
      __syncwarp();
    }
  } else {
    for (int k = 0; k < m; ++k) {              // U^T w = x
      if (lane == 0) x[k] /= LU[k + k * m];
      __syncwarp();
      const double xk = x[k];
      for (int i = k + 1 + lane; i < m; i += 32) x[i] -= LU[k + i * m] * xk;
      __syncwarp();
    }
    for (int k = m - 1; k >= 0; --k) {         // L^T v = w
      const double xk = x[k];
      for (int i = lane; i < k; i += 32) x[i] -= LU[k + i * m] * xk;
      __syncwarp();
    }
    if (lane == 0)                             // x = P^T v: the row swaps undone in reverse
      for (int k = m - 1; k >= 0; --k)
        if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
    __syncwarp();
  }
}

__device__ inline double warp_dot(const double* a, const double* b, int m) {
  double acc = 0.0;
  for (int i = threadIdx.x & 31; i < m; i += 32) acc += a[i] * b[i];
  return warp_sum(acc);
}

// Deflation of the near-null eigenvalues of A = H_m (in place) for a C with capacitor-free
// nodes, where J^-1 = -G^-1 C has the eigenvalue 0 and exp(h H^-1) takes its limit from the
// stable side: an eigenvalue mu0 with |mu0| <= h/700 (e^{h/mu} < 1e-304 for a stiff real
// mode; a tiny one of either sign is the rounding image of a zero) is moved to -h/800, where
// e^{h/mu} = e^-800 is 0 in FP64, by the rank-one Wielandt update
//     A <- A + (-h/800 - mu0) r l^T / (l^T r)
// with r, l its right and left eigenvectors.  l^T is orthogonal to every other right
// eigenvector, so the rest of the spectrum and its eigenvectors are unchanged.  r and l come
// from 8 inverse iterations on the LU of A (pivots floored at 2^-52 max|A| so that an exactly
// singular A still gives a direction), with the already deflated pairs projected out so that
// each pass finds the next smallest eigenvalue; mu0 is the two-sided Rayleigh quotient
// l^T A r / l^T r.  The loop stops at the first eigenvalue above h/700, or when the pair is
// not converged (residual above 1e-8 max|A|, l^T r below 1e-10).  W: m x m scratch, R, Lv:
// m x m (deflated pairs by column), vec: 8 m doubles.
__device__ inline void sm_deflate(double* A, int m, double h, double* W, double* R, double* Lv,
                                  double* vec, int* ipiv) {
  const double tau = h / 700.0, delta = h / 800.0;
  double* x = vec;
  double* y = vec + m;
  double* t = vec + 2 * m;
  double* dk = vec + 3 * m;
  __shared__ double s_nrm, s_mu, s_d;
  __shared__ int s_ok;
  if (threadIdx.x < 32) {
    double mx = 0.0;
    for (int e = threadIdx.x; e < m * m; e += 32) mx = fmax(mx, fabs(A[e]));
    mx = warp_max(mx);
    if (threadIdx.x == 0) s_nrm = mx;
  }
  __syncthreads();
  const double nrm = s_nrm;
  const double floor = fmax(1e-300, 2.220446049250313e-16 * nrm);
  for (int nd = 0; nd < m; ++nd) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) W[e] = A[e];
    __syncthreads();
    sm_lu(W, ipiv, m, floor);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      const double v0 = rsqrt((double)m);
      for (int i = lane; i < m; i += 32) { x[i] = v0; y[i] = v0; }
      __syncwarp();
      for (int it = 0; it < 8; ++it) {
        warp_lu_solve_vec(W, ipiv, x, m, false);
        warp_lu_solve_vec(W, ipiv, y, m, true);
        for (int q = 0; q < nd; ++q) {          // project out the deflated pairs
          const double* rq = R + q * m;
          const double* lq = Lv + q * m;
          const double cx = warp_dot(lq, x, m) / dk[q];
          const double cy = warp_dot(rq, y, m) / dk[q];
          for (int i = lane; i < m; i += 32) { x[i] -= cx * rq[i]; y[i] -= cy * lq[i]; }
          __syncwarp();
        }
        const double nx = sqrt(warp_dot(x, x, m)), ny = sqrt(warp_dot(y, y, m));
        for (int i = lane; i < m; i += 32) { x[i] /= nx; y[i] /= ny; }
        __syncwarp();
      }
      for (int i = lane; i < m; i += 32) {     // t = A x
        double acc = 0.0;
        for (int j = 0; j < m; ++j) acc += A[i + j * m] * x[j];
        t[i] = acc;
      }
      __syncwarp();
      const double d = warp_dot(y, x, m);
      const double mu = warp_dot(y, t, m) / d;
      double res = 0.0;
      for (int i = lane; i < m; i += 32) res = fmax(res, fabs(t[i] - mu * x[i]));
      res = warp_max(res);
      if (lane == 0) {
        s_ok = isfinite(d) && isfinite(mu) && fabs(d) >= 1e-10 && fabs(mu) <= tau &&
               res <= 1e-8 * nrm;
        s_mu = mu;
        s_d = d;
      }
    }
    __syncthreads();
    if (!s_ok) break;
    const double c = (-delta - s_mu) / s_d;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = e % m, j = e / m;
      A[e] += c * x[i] * y[j];
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) { R[nd * m + i] = x[i]; Lv[nd * m + i] = y[i]; }
    if (threadIdx.x == 0) dk[nd] = s_d;
    __syncthreads();
  }
}

// y = exp(h H^-1) e_1 for the leading m x m block of H (ld ldh); last = e_m^T H^-1 y.
// Scaling and squaring of the diagonal [13/13] Pade approximant (theta_13 = 5.37), after the
// deflation of near-null eigenvalues when pade.deflate is set (C with capacitor-free nodes).
// Returns true when y and last are finite.  smem: small_smem_doubles(m) doubles.
template <int CS = 1>
__device__ inline bool phi_small(const double* H, int ldh, int m, double h, double* y,
                                 double* last, double* smem, int* ipiv, const PadeCoef& pade) {
  const double* c_pade = pade.c;
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
  if (pade.deflate) sm_deflate(M0, m, h, M2, M3, M4, vec + m, ipiv);
  __shared__ double s_rd[MAX_M];
  sm_lu(M0, ipiv, m, 0.0, s_rd);
  sm_lu_solve<CS>(M0, ipiv, s_rd, M1, m);    // M1 = X = h H^-1
  for (int k = threadIdx.x; k < m; k += blockDim.x) lastrow[k] = M1[(m - 1) + k * m] / h;
  __shared__ double s_cs[MAX_M];
  for (int jj = threadIdx.x; jj < m; jj += blockDim.x) {   // column sums of |X|, rows in order
    double cs = 0.0;
    for (int i = 0; i < m; ++i) cs += fabs(M1[i + jj * m]);
    s_cs[jj] = cs;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int jj = 0; jj < m; ++jj) nrm = fmax(nrm, s_cs[jj]);
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
  sm_matmul<CS>(M2, M1, M1, m);   // A2
  sm_matmul<CS>(M3, M2, M2, m);   // A4
  sm_matmul<CS>(M4, M3, M2, m);   // A6
  for (int e = threadIdx.x; e < m * m; e += blockDim.x)
    M0[e] = c_pade[13] * M4[e] + c_pade[11] * M3[e] + c_pade[9] * M2[e];
  __syncthreads();
  sm_matmul<CS>(M5, M4, M0, m);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, jj = e / m;
    M5[e] += c_pade[7] * M4[e] + c_pade[5] * M3[e] + c_pade[3] * M2[e] + (i == jj ? c_pade[1] : 0.0);
  }
  __syncthreads();
  sm_matmul<CS>(M0, M1, M5, m);   // U
  for (int e = threadIdx.x; e < m * m; e += blockDim.x)
    M5[e] = c_pade[12] * M4[e] + c_pade[10] * M3[e] + c_pade[8] * M2[e];
  __syncthreads();
  sm_matmul<CS>(M1, M4, M5, m);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int i = e % m, jj = e / m;
    double V = M1[e] + c_pade[6] * M4[e] + c_pade[4] * M3[e] + c_pade[2] * M2[e] +
               (i == jj ? c_pade[0] : 0.0);
    M2[e] = V - M0[e];
    M3[e] = V + M0[e];
  }
  __syncthreads();
  sm_lu(M2, ipiv, m, 0.0, s_rd);
  sm_lu_solve<CS>(M2, ipiv, s_rd, M3, m);   // R = (V - U)^-1 (V + U)
  double* R = M3;
  double* Tm = M4;
  for (int q = 0; q + 1 < s; ++q) {
    sm_matmul<CS>(Tm, R, R, m);
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



// The decision of Algorithm 1 for one Krylov space after its latest Arnoldi iteration
// (mode RESID), at the end of a fixed-dimension run (FIXED_END), or for an existing basis at
// a new h (FINAL).  Writes y = exp(h H_m^-1) e_1 and m into the space's state.
//
// m_first (>= m_min) is the dimension at which the first decision is taken; the plain rule
// has m_first = m_min.  A larger m_first (a proposed dimension) skips the tests below it.
// When the basis reaches m_first the space is flagged (K.scan) and the caller tests the
// dimensions [m_min, m_first] in parallel, taking the first that passes; if the basis breaks
// down before m_first, the skipped dimensions are tested here in increasing order.  Either way
// the chosen dimension is the one the plain rule picks, and never a larger one: past its
// converged dimension a basis gathers rounding-noise directions whose spurious Ritz values
// can pass the residual test with a wrong exp(h H^-1) e_1.
template <int CS = 1>
__device__ inline void small_decide(int mode, const double* H, KrylovState& K, double h,
                                    double eps, int m_min, int m_max, int m_first, double* smem,
                                    int* ipiv, double* ybuf, double* s_last, unsigned* status,
                                    const PadeCoef& pade) {
  const int ldh = MAX_M + 1;
  __shared__ int s_done, s_m, s_built, s_bd, s_m_in, s_conv;
  if (threadIdx.x == 0) {
    s_done = K.done; s_m = K.m; s_built = K.built; s_bd = K.breakdown;
    s_m_in = (K.beta > 0.0);
  }
  __syncthreads();
  if (!s_m_in) return;   // zero vector: MEVP = 0
  auto write_y = [&](int m) {
    for (int k = threadIdx.x; k < m; k += blockDim.x) K.y[k] = ybuf[k];
    if (threadIdx.x == 0) { K.last = *s_last; K.m = m; }
  };
  // residual test (Eq. 16) at dimension jj <= built; true (and y written, space done) if it
  // passes.  Tracks the smallest finite residual.
  auto test_dim = [&](int jj) -> bool {
    bool fin = phi_small<CS>(H, ldh, jj, h, ybuf, s_last, smem, ipiv, pade);
    if (threadIdx.x == 0) {
      double res = H[jj + (jj - 1) * ldh] * K.gvnext[jj - 1] * fabs(*s_last) / K.gv1;
      if (!fin) res = INFINITY;
      K.res = res;
      if (isfinite(res) && res < K.best_res) { K.best_res = res; K.best_m = jj; }
      s_conv = isfinite(res) && res < eps;
    }
    __syncthreads();
    if (s_conv) {
      write_y(jj);
      if (threadIdx.x == 0) K.done = 1;
    }
    __syncthreads();
    return s_conv;
  };
  // the skipped dimensions [m_min, hi] in increasing order
  auto scan_skipped = [&](int hi) -> bool {
    for (int jj = m_min; jj <= hi; ++jj)
      if (test_dim(jj)) return true;
    return false;
  };
  // dimension at a breakdown: built, or built-1 when the last direction was noise
  auto finalize_breakdown = [&]() {
    int m = s_built;
    bool fin = phi_small<CS>(H, ldh, m, h, ybuf, s_last, smem, ipiv, pade);
    if (!fin && m > 1) {
      m -= 1;
      fin = phi_small<CS>(H, ldh, m, h, ybuf, s_last, smem, ipiv, pade);
    }
    if (!fin && threadIdx.x == 0) atomicOr(status, ST_KRYLOV);
    write_y(m);
  };
  if (mode == SMALL_FINAL) {
    bool fin = phi_small<CS>(H, ldh, s_m, h, ybuf, s_last, smem, ipiv, pade);
    if (!fin && threadIdx.x == 0) atomicOr(status, ST_KRYLOV);
    write_y(s_m);
    return;
  }
  if (mode == SMALL_FIXED_END) {
    if (s_bd) { finalize_breakdown(); return; }
    bool fin = phi_small<CS>(H, ldh, s_built, h, ybuf, s_last, smem, ipiv, pade);
    if (!fin && threadIdx.x == 0) atomicOr(status, ST_KRYLOV);
    write_y(s_built);
    if (threadIdx.x == 0) K.done = 1;
    return;
  }
  // SMALL_RESID: called after every Arnoldi iteration in adaptive mode
  m_first = max(m_first, m_min);
  if (s_done && !s_bd) return;   // already converged earlier
  if (s_bd) {
    if (s_m == s_built) {
      if (m_first > m_min && s_built <= m_first && scan_skipped(s_built - 1)) {
        if (threadIdx.x == 0) K.breakdown = 2;
        return;
      }
      finalize_breakdown();
      if (threadIdx.x == 0) K.breakdown = 2;
    }
    return;
  }
  int jj = s_built;
  if (m_first > m_min && jj == m_first) {
    if (threadIdx.x == 0) K.scan = 1;   // [m_min, m_first] are tested in parallel by the caller
    return;
  }
  if (jj >= m_first && jj >= m_min && test_dim(jj)) return;
  if (jj >= m_max) {
    // never converged: the dimension with the smallest finite residual; when no tested
    // dimension had one, the largest dimension whose exp(h H^-1) e_1 is finite
    int m = K.best_m > 0 ? K.best_m : jj;
    __syncthreads();
    bool fin = phi_small<CS>(H, ldh, m, h, ybuf, s_last, smem, ipiv, pade);
    while (!fin && m > 1) {
      --m;
      fin = phi_small<CS>(H, ldh, m, h, ybuf, s_last, smem, ipiv, pade);
    }
    if (!fin && threadIdx.x == 0) atomicOr(status, ST_KRYLOV);
    write_y(m);
    if (threadIdx.x == 0) K.done = 1;
  }
}

}  // namespace ers
