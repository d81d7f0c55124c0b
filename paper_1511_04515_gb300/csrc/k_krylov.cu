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
#include "kdense.cuh"

namespace ers {

constexpr int KB = 256;          // threads per block of the vector kernels


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

struct SmallArgs {
  PadeCoef pade;
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
  if (A.mode == SMALL_TEST) {
    phi_small(A.Htest, A.ldh_test, A.m_test, A.h, ybuf, &s_last, smem, ipiv, A.pade);
    for (int k = threadIdx.x; k < A.m_test; k += blockDim.x) A.y_out[k] = ybuf[k];
    if (threadIdx.x == 0) *A.last_out = s_last;
    return;
  }
  int b = blockIdx.x;
  small_decide(A.mode, A.H[b], A.ks[A.slot[b]], A.h, A.eps, A.m_min, A.m_max, A.m_min, smem, ipiv, ybuf,
               &s_last, A.status, A.pade);
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
  return cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              small_smem_doubles(MAX_M) * 8);
}

// Grid of the cooperative vector kernels: every inner product of MGS is a grid-wide reduction
// (arrival counter, one CTA sums the partials), whose cost grows with the CTA count, so the grid
// is sized for at least 8 elements per thread; the memory traffic of an iteration stays far
// below what the resulting CTAs can stream.
static int coop_blocks_for(ers_ctx* c, int n) {
  int want = (n + 8 * KB - 1) / (8 * KB);
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
  A.pade = pade_coefficients(c->singular_c);
  A.mode = mode;
  A.nb = g.nb;
  for (int b = 0; b < g.nb; ++b) { A.slot[b] = g.slot[b]; A.H[b] = g.H[b]; }
  A.ks = c->ks;
  A.h = h;
  A.eps = c->opts.eps_krylov;
  A.m_min = c->opts.m_min;
  A.m_max = m_max;
  A.status = c->d_status;
  size_t sm = small_smem_doubles((size_t)c->opts.m_max) * 8;
  k_small<<<g.nb, KB, sm, c->stream>>>(A);
  c->stats.kernel_launches++;
  return cudaGetLastError();
}

cudaError_t launch_small_test(ers_ctx* c, const double* H, int ldh, int m, double h, double* y,
                              double* last) {
  SmallArgs A{};
  A.pade = pade_coefficients(c->singular_c);
  A.mode = SMALL_TEST;
  A.h = h;
  A.Htest = H;
  A.ldh_test = ldh;
  A.m_test = m;
  A.y_out = y;
  A.last_out = last;
  size_t sm = small_smem_doubles((size_t)m) * 8;
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
