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
#include <mutex>

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
  double* part;         // grid-reduction partials: 2 * GRID_RED_NV * gridDim
  unsigned* bar;        // arrival / exit counters of the grid reductions
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

// NB: number of spaces in the group (compile-time, so that per-space values stay in registers)
template <int NB>
__global__ void __launch_bounds__(KB) k_arnoldi_init(CoopArgs A) {
  __shared__ double sh[GRID_RED_NV * (KB / 32)];
  GridRed gr{A.part, A.bar, A.status, 0u};
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double beta[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    double acc = 0.0;
    for (int64_t i = tid; i < A.n; i += T) { double v = A.g.src[b][i]; acc += v * v; }
    beta[b] = acc;
  }
  grid_sum_n<NB>(beta, gr, sh);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    beta[b] = sqrt(beta[b]);
    double inv = beta[b] > 0.0 ? 1.0 / beta[b] : 0.0;
    for (int64_t i = tid; i < A.n; i += T) A.g.V[b][i] = A.g.src[b][i] * inv;
  }
  double gl[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) gl[b] = 0.0;
  if (A.adaptive) {
    grid_sync(gr);                                   // V_0 complete
#pragma unroll
    for (int b = 0; b < NB; ++b) gl[b] = gnorm_part(A, A.g.V[b], T);
    grid_sum_n<NB>(gl, gr, sh);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      KrylovState& K = A.ks[A.g.slot[b]];
      K.beta = beta[b];
      K.gv1 = A.adaptive ? sqrt(gl[b]) : 0.0;
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
  grid_exit(gr);
}

// One modified Gram-Schmidt step of Algorithm 1 for NB spaces: w = J^-1 v_j (the solve's
// output, negated) is orthogonalised against v_0 .. v_j one vector at a time.  Each thread
// owns EPT elements, at i = tid + q T: w stays in registers, and so does the basis vector of
// the current projection, which is also the one of the next inner product.  With PF the
// vector after it is loaded before the inner product's grid reduction, so the load is in
// flight while the blocks wait for each other (used where the three register arrays fit).
template <int NB, int EPT, bool PF>
__global__ void __launch_bounds__(KB, 2) k_mgs(CoopArgs A) {
  __shared__ double sh[GRID_RED_NV * (KB / 32)];
  GridRed gr{A.part, A.bar, A.status, 0u};
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int j = A.j, n = A.n;
  constexpr int ldh = MAX_M + 1;
  bool active[NB], any = false;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    active[b] = !A.ks[A.g.slot[b]].done;
    any = any || active[b];
  }
  // every space finished (a launch the host queued before it knew): nothing to do.  The
  // flags come from earlier launches, so every block returns here, before any reduction.
  if (!any) return;
  // PF: cur = v_i and nxt = v_{i+1} in registers; otherwise both are read at their use
  double w[NB][EPT], cur[NB][EPT], nxt[NB][EPT];
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int64_t i = tid + q * T;
      w[b][q] = (active[b] && i < n) ? -A.g.src[b][i] : 0.0;
      cur[b][q] = (PF && i < n) ? A.g.V[b][i] : 0.0;
      nxt[b][q] = 0.0;
    }
  if (PF && j >= 1)
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int64_t i = tid + q * T;
        nxt[b][q] = i < n ? A.g.V[b][(int64_t)n + i] : 0.0;
      }
  // pass 0: ||w||^2 and <w, v_0>
  double r0[2 * NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    double nn = 0.0, dd = 0.0;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int64_t i = tid + q * T;
      const double v0 = PF ? cur[b][q] : (i < n ? A.g.V[b][i] : 0.0);
      nn += w[b][q] * w[b][q];
      dd += w[b][q] * v0;
    }
    r0[2 * b] = nn;
    r0[2 * b + 1] = dd;
  }
  grid_sum_n<2 * NB>(r0, gr, sh);
  double w0[NB], hcur[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) { w0[b] = sqrt(r0[2 * b]); hcur[b] = r0[2 * b + 1]; }
  if (blockIdx.x == 0 && threadIdx.x == 0)
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (active[b]) A.g.H[b][0 + j * ldh] = hcur[b];
  for (int i = 0; i <= j; ++i) {
    double lp[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int64_t e = tid + q * T;
        const double vi = PF ? cur[b][q] : (e < n ? A.g.V[b][(int64_t)i * n + e] : 0.0);
        w[b][q] -= hcur[b] * vi;
        if (i < j) {
          const double v = PF ? nxt[b][q] : (e < n ? A.g.V[b][(int64_t)(i + 1) * n + e] : 0.0);
          acc += w[b][q] * v;
          if (PF) cur[b][q] = v;
        } else {
          acc += w[b][q] * w[b][q];
        }
      }
      lp[b] = acc;
    }
    if (PF && i + 1 < j)                 // v_{i+2}, in flight during the reduction
#pragma unroll
      for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
          const int64_t e = tid + q * T;
          nxt[b][q] = e < n ? A.g.V[b][(int64_t)(i + 2) * n + e] : 0.0;
        }
    grid_sum_n<NB>(lp, gr, sh);
#pragma unroll
    for (int b = 0; b < NB; ++b) hcur[b] = lp[b];
    if (i < j && blockIdx.x == 0 && threadIdx.x == 0)
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (active[b]) A.g.H[b][(i + 1) + j * ldh] = hcur[b];
  }
  // hcur = ||w||^2 after orthogonalisation
  double hn[NB];
  bool bd[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    hn[b] = sqrt(hcur[b]);
    bd[b] = !(hn[b] > 1e-12 * w0[b]);
    if (!active[b] || bd[b]) continue;
    const double inv = 1.0 / hn[b];
    double* vn = A.g.V[b] + (int64_t)(j + 1) * n;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int64_t e = tid + q * T;
      if (e < n) vn[e] = w[b][q] * inv;
    }
  }
  double gl[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) gl[b] = 0.0;
  if (A.adaptive) {
    grid_sync(gr);                                   // v_{j+1} complete
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (active[b] && !bd[b]) gl[b] = gnorm_part(A, A.g.V[b] + (int64_t)(j + 1) * n, T);
    grid_sum_n<NB>(gl, gr, sh);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (!active[b]) continue;
      KrylovState& K = A.ks[A.g.slot[b]];
      A.g.H[b][(j + 1) + j * ldh] = hn[b];
      K.w0 = w0[b];
      K.built = j + 1;
      K.gvnext[j] = A.adaptive && !bd[b] ? sqrt(gl[b]) : 0.0;
      if (!isfinite(hn[b])) atomicOr(A.status, ST_NONFINITE);
      if (bd[b]) { K.breakdown = 1; K.done = 1; K.m = j + 1; }
    }
  }
  grid_exit(gr);
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

// One space per cluster of SMALL_CS CTAs (kdense.cuh: every CTA computes a column slab of
// each product and holds the whole result).  The CTA of rank 0 works on the space's state in
// global memory; the others on a shared-memory copy that they update identically, so every
// CTA takes the same branches and only rank 0 writes results.
constexpr int SMALL_CS = 8;

__global__ void __cluster_dims__(SMALL_CS, 1, 1) k_small(SmallArgs A) {
  extern __shared__ double smem[];
  __shared__ int ipiv[MAX_M];
  __shared__ double ybuf[MAX_M];
  __shared__ double s_last;
  __shared__ KrylovState kcopy;
  const unsigned rank = cl_rank();
  if (A.mode == SMALL_TEST) {
    phi_small<SMALL_CS>(A.Htest, A.ldh_test, A.m_test, A.h, ybuf, &s_last, smem, ipiv, A.pade);
    if (rank == 0) {
      for (int k = threadIdx.x; k < A.m_test; k += blockDim.x) A.y_out[k] = ybuf[k];
      if (threadIdx.x == 0) *A.last_out = s_last;
    }
    return;
  }
  const int b = blockIdx.x / SMALL_CS;
  KrylovState* K = A.ks + A.slot[b];
  if (rank != 0) {
    const int* src = reinterpret_cast<const int*>(K);
    int* dst = reinterpret_cast<int*>(&kcopy);
    for (int e = threadIdx.x; e < (int)(sizeof(KrylovState) / sizeof(int)); e += blockDim.x)
      dst[e] = src[e];
    __syncthreads();
    K = &kcopy;
  }
  small_decide<SMALL_CS>(A.mode, A.H[b], *K, A.h, A.eps, A.m_min, A.m_max, A.m_min, smem, ipiv,
                         ybuf, &s_last, A.status, A.pade);
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
// whose latency grows with the CTA count, so the grid is sized for about 8 elements per thread
// (one CTA up to 2,048 nodes); the memory traffic of an iteration stays far below what the
// resulting CTAs can stream.
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
  A.bar = c->d_status + 4;
  A.status = c->d_status;
  return A;
}

typedef void (*CoopKernel)(CoopArgs);

// Krylov groups hold one or two spaces (the solution bases of a ramp step, or one basis)
constexpr int MGS_MAX_NB = 2;

static CoopKernel init_kernel(int nb) { return nb == 1 ? k_arnoldi_init<1> : k_arnoldi_init<2>; }

constexpr int EPT_LEVELS = 5;     // 1, 2, 4, 8, 16 elements per thread

// the prefetching variant exists where its three register arrays (NB x EPT doubles each) fit
static bool pf_exists(int nb, int lvl) { return nb * (1 << lvl) <= 16; }

template <int NB, int EPT, bool PF>
static CoopKernel mgs_instance() {
  if constexpr (PF && NB * EPT > 16) return nullptr;
  else return k_mgs<NB, EPT, PF>;
}

template <int NB, bool PF>
static CoopKernel mgs_kernel_nb(int lvl) {
  switch (lvl) {
    case 0: return mgs_instance<NB, 1, PF>();
    case 1: return mgs_instance<NB, 2, PF>();
    case 2: return mgs_instance<NB, 4, PF>();
    case 3: return mgs_instance<NB, 8, PF>();
    default: return mgs_instance<NB, 16, PF>();
  }
}

static CoopKernel mgs_kernel(int nb, int lvl, bool pf) {
  if (pf) return nb == 1 ? mgs_kernel_nb<1, true>(lvl) : mgs_kernel_nb<2, true>(lvl);
  return nb == 1 ? mgs_kernel_nb<1, false>(lvl) : mgs_kernel_nb<2, false>(lvl);
}

// resident CTAs per SM of the prefetching MGS variants (0 where a variant does not exist)
static int g_pf_occ[MGS_MAX_NB][EPT_LEVELS];
static std::once_flag g_pf_once;

static void pf_occupancy() {
  for (int nb = 1; nb <= MGS_MAX_NB; ++nb)
    for (int l = 0; l < EPT_LEVELS; ++l) {
      int occ = 0;
      if (pf_exists(nb, l))
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mgs_kernel(nb, l, true), KB, 0);
      g_pf_occ[nb - 1][l] = occ;
    }
}

cudaError_t launch_arnoldi_init(ers_ctx* c, const VecGroup& g, int adaptive) {
  if (g.nb < 1 || g.nb > MGS_MAX_NB) return cudaErrorInvalidValue;
  CoopArgs A = make_coop(c, g, 0, adaptive);
  int blocks = coop_blocks_for(c, c->n);
  void* args[] = {&A};
  c->stats.kernel_launches++;
  return cudaLaunchCooperativeKernel((void*)init_kernel(g.nb), blocks, KB, args, 0, c->stream);
}

cudaError_t launch_mgs(ers_ctx* c, const VecGroup& g, int j, int adaptive) {
  if (g.nb < 1 || g.nb > MGS_MAX_NB) return cudaErrorInvalidValue;
  CoopArgs A = make_coop(c, g, j, adaptive);
  const int blocks = coop_blocks_for(c, c->n);
  const int64_t T = (int64_t)blocks * KB;
  const int64_t ept = (c->n + T - 1) / T;
  int lvl = 0;
  while (lvl < EPT_LEVELS && ((int64_t)1 << lvl) < ept) ++lvl;
  if (lvl >= EPT_LEVELS) return cudaErrorInvalidValue;
  std::call_once(g_pf_once, pf_occupancy);
  const bool pf = pf_exists(g.nb, lvl) && (int64_t)g_pf_occ[g.nb - 1][lvl] * c->sm_count >= blocks;
  void* args[] = {&A};
  c->stats.kernel_launches++;
  return cudaLaunchCooperativeKernel((void*)mgs_kernel(g.nb, lvl, pf), blocks, KB, args, 0,
                                     c->stream);
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
  k_small<<<g.nb * SMALL_CS, KB, sm, c->stream>>>(A);
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
  k_small<<<SMALL_CS, KB, sm, c->stream>>>(A);
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

// Co-resident CTAs of the cooperative kernels: the smallest count over the Arnoldi start and
// the non-prefetching MGS variants at 16 elements per thread (the launch falls back to those),
// at most 4 per SM.
int coop_max_blocks(int sm_count) {
  int per_sm = 4;
  for (int nb = 1; nb <= MGS_MAX_NB; ++nb) {
    int o1 = 0, o2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, mgs_kernel(nb, EPT_LEVELS - 1, false), KB, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, init_kernel(nb), KB, 0);
    per_sm = std::min(per_sm, std::min(o1, o2));
  }
  // the reduction scratch holds 2 * GRID_RED_NV partials per block in 2 * MAX_RHS * 4096 doubles
  return std::max(1, std::min(per_sm * sm_count, MAX_RHS * 4096 / GRID_RED_NV));
}

}  // namespace ers
