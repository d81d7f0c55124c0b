// Device evaluation, stamping of G_k and F_k, and the numeric LU refactor of G_k.
//
// Alg. 2 derives G_k and F_k from the device models at x_k and factors G_k once per step
// (never C, never C/h + G).  The LU reuses the pattern analysed once on the host and runs
// as a level-scheduled multifrontal factorisation with static pivots:
//   per level (leaves first): zero fronts -> scatter A -> extend-add children ->
//   factor the w x w pivot block (and invert its L and U for the solves) ->
//   scale the panels (F21 U11^-1, L11^-1 F12) -> Schur update F22 -= F21 F12.
#include "ers_internal.h"
#include "kcommon.cuh"

namespace ers {

// ---------------------------------------------------------------------------------------
// Square-law MOSFET (stand-in for BSIM3): current d -> s and partials w.r.t. (vd, vg, vs).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void nmos_forward(double vgs, double vds, double vt, double k,
                                             double lam, double& I, double& gm, double& gds) {
  double vov = vgs - vt;
  if (vov <= 0.0) { I = 0.0; gm = 0.0; gds = 0.0; return; }
  double clm = 1.0 + lam * vds;
  if (vds < vov) {
    double core = vov * vds - 0.5 * vds * vds;
    I = k * core * clm;
    gm = k * vds * clm;
    gds = k * (vov - vds) * clm + k * core * lam;
  } else {
    double core = 0.5 * vov * vov;
    I = k * core * clm;
    gm = k * vov * clm;
    gds = k * core * lam;
  }
}

__device__ __forceinline__ void mosfet_eval(int type, double vd, double vg, double vs,
                                            double vt, double k, double lam, double& ids,
                                            double& dd, double& dg, double& ds) {
  double sgn = 1.0;
  if (type == 1) { vd = -vd; vg = -vg; vs = -vs; sgn = -1.0; }
  double I, gm, gds;
  if (vd >= vs) {
    nmos_forward(vg - vs, vd - vs, vt, k, lam, I, gm, gds);
    ids = I; dd = gds; dg = gm; ds = -gm - gds;
  } else {
    nmos_forward(vg - vd, vs - vd, vt, k, lam, I, gm, gds);
    ids = -I; dd = gm + gds; dg = -gm; ds = -gds;
  }
  ids *= sgn;
}

__device__ __forceinline__ double term_v(int node, const double* x, double vdd) {
  return node >= 0 ? x[node] : (node == -1 ? 0.0 : vdd);
}

// dev_I[d] = current at x; with_jac: dev_J[3d..3d+2] = partials.
__global__ void k_dev_eval(int ndev, const int32_t* type, const int32_t* term,
                           const double* par, const double* x, double vdd, double* dev_I,
                           double* dev_J, int with_jac) {
  int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= ndev) return;
  int tn = term[3 * d], tg = term[3 * d + 1], ts = term[3 * d + 2];
  double ids, dd, dg, ds;
  mosfet_eval(type[d], term_v(tn, x, vdd), term_v(tg, x, vdd), term_v(ts, x, vdd),
              par[3 * d], par[3 * d + 1], par[3 * d + 2], ids, dd, dg, ds);
  dev_I[d] = ids;
  if (with_jac) {
    dev_J[3 * d] = dd;
    dev_J[3 * d + 1] = dg;
    dev_J[3 * d + 2] = ds;
  }
}

// G_k values at every slot of the union pattern: linear value plus the device partials
// that land on the slot (gather list per slot: entry = dev*8 + which*2 + negative).
__global__ void k_stamp(int nnz, const double* Glin, const int32_t* sptr, const int32_t* sent,
                        const double* dev_J, double* Gval) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  double v = Glin[e];
  for (int q = sptr[e]; q < sptr[e + 1]; ++q) {
    int code = sent[q];
    double j = dev_J[3 * (code >> 3) + ((code >> 1) & 3)];
    v += (code & 1) ? -j : j;
  }
  Gval[e] = v;
}

// Per node i, over incident devices (entry = dev*2 + negative):
//   mode 0: F_i  = sum sign * (J_k . x_nonrail - I_k)                 (F_k at x_k)
//   mode 1: dF_i = sum sign * (J_k . (xn - xk)_nonrail - (I_new - I_k)) (F(x_new) - F_k)
__global__ void k_node_F(int n, const int32_t* nptr, const int32_t* nent, const int32_t* term,
                         const double* dev_J, const double* dev_I, const double* dev_In,
                         const double* xk, const double* xn, int mode, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int q = nptr[i]; q < nptr[i + 1]; ++q) {
    int code = nent[q];
    int d = code >> 1;
    double lin = 0.0;
    for (int t = 0; t < 3; ++t) {
      int node = term[3 * d + t];
      if (node >= 0) {
        double xv = mode == 0 ? xk[node] : (xn[node] - xk[node]);
        lin += dev_J[3 * d + t] * xv;
      }
    }
    double cur = mode == 0 ? dev_I[d] : (dev_In[d] - dev_I[d]);
    double c = lin - cur;
    acc += (code & 1) ? -c : c;
  }
  out[i] = acc;
}

// ---------------------------------------------------------------------------------------
// Multifrontal refactor kernels.  Front of supernode s: f x f column-major at
// arena + front_off[s], f = w + r, rows/cols = [own columns, R_off(s)].
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void sn_dims(const DevicePlan& P, int s, int& c0, int& w, int& r) {
  c0 = P.sn_start[s];
  w = P.sn_start[s + 1] - c0;
  r = (int)(P.rptr[s + 1] - P.rptr[s]);
}

__global__ void k_mf_zero(DevicePlan P, int lo, int hi) {
  int s = P.lvl_sn[lo + blockIdx.x];
  int c0, w, r;
  sn_dims(P, s, c0, w, r);
  int64_t f = w + r, sz = f * f;
  double* F = P.arena + P.front_off[s];
  int64_t stride = (int64_t)gridDim.y * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x; e < sz; e += stride) F[e] = 0.0;
}

__global__ void k_mf_assemble(DevicePlan P, int lo, int hi, const double* Gval) {
  int k = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= hi) return;
  int e = P.lvl_slot[k];
  P.arena[P.asm_dst[e]] = Gval[e];
}

// extend-add of every child into the supernodes lvl_sn[lo..hi) in one launch: CTA (x, y)
// owns the columns pcol of parent lvl_sn[lo + x] with pcol % gridDim.y == y and adds the
// parent's children one after another in rank order (a barrier between children, whose rows
// reach the same parent entries through different threads).  Every parent entry thus receives
// its additions in the same order as with one launch per child rank: the same sums, bit for
// bit, and no two CTAs write one entry.
__global__ void k_mf_extend_add_level(DevicePlan P, int lo) {
  const int p = P.lvl_sn[lo + blockIdx.x];
  const int cb = P.ch_ptr[p], ce = P.ch_ptr[p + 1];
  if (cb == ce) return;
  int pc0, pw, pr;
  sn_dims(P, p, pc0, pw, pr);
  const int64_t fp = pw + pr;
  double* Fp = P.arena + P.front_off[p];
  for (int q = cb; q < ce; ++q) {
    const int c = P.ch_list[q];
    int cc0, cw, cr;
    sn_dims(P, c, cc0, cw, cr);
    const int64_t fc = cw + cr;
    const double* Fc = P.arena + P.front_off[c];
    const int32_t* rel = P.rel + P.rptr[c];
    for (int b = 0; b < cr; ++b) {
      const int pcol = rel[b];
      if (pcol % (int)gridDim.y != (int)blockIdx.y) continue;
      const double* src = Fc + (int64_t)(cw + b) * fc + cw;
      double* dst = Fp + (int64_t)pcol * fp;
      for (int a = threadIdx.x; a < cr; a += blockDim.x) dst[rel[a]] += src[a];
    }
    __syncthreads();
  }
}

// Factor the w x w pivot block of each supernode of the level in shared memory
// (no pivoting), write it back, and store L11^-1 (unit lower) and U11^-1.
__global__ void k_mf_diag(DevicePlan P, int lo, unsigned* status) {
  extern __shared__ double sm[];
  int s = P.lvl_sn[lo + blockIdx.x];
  int c0, w, r;
  sn_dims(P, s, c0, w, r);
  int64_t f = w + r;
  double* F = P.arena + P.front_off[s];
  double* A = sm;            // w x w, ld w
  double* X = sm + w * w;    // inverse workspace
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) A[e] = F[(e % w) + (int64_t)(e / w) * f];
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    double piv = A[k + k * w];
    if (threadIdx.x == 0 && (!(fabs(piv) > 1e-300) || !isfinite(piv))) atomicOr(status, ST_SINGULAR);
    double inv = 1.0 / piv;
    for (int i = k + 1 + threadIdx.x; i < w; i += blockDim.x) A[i + k * w] *= inv;
    __syncthreads();
    int rem = w - k - 1;
    for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      int i = k + 1 + e % rem, j = k + 1 + e / rem;
      A[i + j * w] -= A[i + k * w] * A[k + j * w];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) F[(e % w) + (int64_t)(e / w) * f] = A[e];
  // L11^-1: column j by thread j (forward substitution on the unit lower factor)
  for (int j = threadIdx.x; j < w; j += blockDim.x) {
    for (int i = 0; i < j; ++i) X[i + j * w] = 0.0;
    X[j + j * w] = 1.0;
    for (int i = j + 1; i < w; ++i) {
      double acc = 0.0;
      for (int q = j; q < i; ++q) acc += A[i + q * w] * X[q + j * w];
      X[i + j * w] = -acc;
    }
  }
  __syncthreads();
  double* LDi = P.LDi + P.d_off[s];
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) LDi[e] = X[e];
  __syncthreads();
  // U11^-1: column j by thread j (back substitution)
  for (int j = threadIdx.x; j < w; j += blockDim.x) {
    for (int i = j + 1; i < w; ++i) X[i + j * w] = 0.0;
    X[j + j * w] = 1.0 / A[j + j * w];
    for (int i = j - 1; i >= 0; --i) {
      double acc = 0.0;
      for (int q = i + 1; q <= j; ++q) acc += A[i + q * w] * X[q + j * w];
      X[i + j * w] = -acc / A[i + i * w];
    }
  }
  __syncthreads();
  double* UDi = P.UDi + P.d_off[s];
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) UDi[e] = X[e];
}

// Panel task (s, r0): rows r0..r0+127 of F21 <- F21 U11^-1 and columns of F12 <- L11^-1 F12;
// results are written back into the front and copied out to Lo / Uo (r x w col-major).
__global__ void k_mf_panel(DevicePlan P, int lo) {
  extern __shared__ double sm[];
  int task = lo + blockIdx.x;
  int s = P.ptask_sn[task], r0 = P.ptask_r0[task];
  int c0, w, r;
  sn_dims(P, s, c0, w, r);
  int64_t f = w + r;
  double* F = P.arena + P.front_off[s];
  const double* LDi = P.LDi + P.d_off[s];
  const double* UDi = P.UDi + P.d_off[s];
  double* sL = sm;            // w x w
  double* sU = sm + w * w;    // w x w
  double* row = sm + 2 * w * w;  // 128 x (w+1) staging
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) { sL[e] = LDi[e]; sU[e] = UDi[e]; }
  int nr = min(128, r - r0);
  const int ld = w + 1;
  double* Lo = P.Lo + P.o_off[s];
  double* Uo = P.Uo + P.o_off[s];
  // F21 rows: load, multiply by U11^-1 (upper), store
  for (int e = threadIdx.x; e < nr * w; e += blockDim.x) {
    int a = e % nr, k = e / nr;
    row[a * ld + k] = F[(w + r0 + a) + (int64_t)k * f];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * w; e += blockDim.x) {
    int a = e % nr, k = e / nr;
    double acc = 0.0;
    for (int j = 0; j <= k; ++j) acc += row[a * ld + j] * sU[j + k * w];
    F[(w + r0 + a) + (int64_t)k * f] = acc;
    Lo[(r0 + a) + (int64_t)k * r] = acc;
  }
  __syncthreads();
  // F12 columns: load (k, a) = F[k + (w + r0 + a) f], multiply by L11^-1 (unit lower)
  for (int e = threadIdx.x; e < nr * w; e += blockDim.x) {
    int k = e % w, a = e / w;
    row[a * ld + k] = F[k + (int64_t)(w + r0 + a) * f];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * w; e += blockDim.x) {
    int k = e % w, a = e / w;
    double acc = 0.0;
    for (int j = 0; j <= k; ++j) acc += sL[k + j * w] * row[a * ld + j];
    F[k + (int64_t)(w + r0 + a) * f] = acc;
    Uo[(r0 + a) + (int64_t)k * r] = acc;
  }
}

// Schur update tile (s, ti, tj): F22[ti*64.., tj*64..] -= F21[ti rows] * F12[tj cols]
__global__ void __launch_bounds__(256) k_mf_schur(DevicePlan P, int lo) {
  extern __shared__ double smem_schur[];
  double (*sA)[65] = reinterpret_cast<double (*)[65]>(smem_schur);             // [k][row]
  double (*sB)[65] = reinterpret_cast<double (*)[65]>(smem_schur + 64 * 65);   // [k][col]
  int task = lo + blockIdx.x;
  int s = P.tile_sn[task];
  int ti = P.tile_ij[task] >> 16, tj = P.tile_ij[task] & 0xffff;
  int c0, w, r;
  sn_dims(P, s, c0, w, r);
  int64_t f = w + r;
  double* F = P.arena + P.front_off[s];
  int i0 = ti * 64, j0 = tj * 64;
  int ni = min(64, r - i0), nj = min(64, r - j0);
  for (int e = threadIdx.x; e < 64 * w; e += blockDim.x) {
    int a = e % 64, k = e / 64;
    sA[k][a] = a < ni ? F[(w + i0 + a) + (int64_t)k * f] : 0.0;
  }
  for (int e = threadIdx.x; e < 64 * w; e += blockDim.x) {
    int k = e % w, b = e / w;
    sB[k][b] = b < nj ? F[k + (int64_t)(w + j0 + b) * f] : 0.0;
  }
  __syncthreads();
  int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k = 0; k < w; ++k) {
    double av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) av[a] = sA[k][tx + 16 * a];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = sB[k][ty + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    int jj = ty + 16 * b;
    if (jj >= nj) continue;
    double* col = F + (int64_t)(w + j0 + jj) * f + w + i0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int ii = tx + 16 * a;
      if (ii < ni) col[ii] -= acc[a][b];
    }
  }
}

// ---------------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------------
void launch_dev_eval(ers_ctx* c, const double* x, double* dev_I, int with_jac) {
  if (!c->ndev) return;
  k_dev_eval<<<(c->ndev + 127) / 128, 128, 0, c->stream>>>(
      c->ndev, c->dev_type, c->dev_term, c->dev_par, x, c->opts.vdd, dev_I, c->dev_J, with_jac);
  c->stats.kernel_launches++;
}

void launch_stamp(ers_ctx* c) {
  k_stamp<<<(c->nnzG + 255) / 256, 256, 0, c->stream>>>(c->nnzG, c->Glin_val, c->stamp_ptr,
                                                          c->stamp_ent, c->dev_J, c->G_val);
  c->stats.kernel_launches++;
}

void launch_node_F(ers_ctx* c, int mode, const double* dev_In, const double* xn, double* out) {
  k_node_F<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->n, c->node_ptr, c->node_ent,
                                                        c->dev_term, c->dev_J, c->dev_I, dev_In,
                                                        c->xk, xn, mode, out);
  c->stats.kernel_launches++;
}

cudaError_t launch_refactor(ers_ctx* c) {
  const Symbolic& S = c->sym;
  DevicePlan& P = c->plan;
  static_assert(MAX_M <= 64, "");
  for (int l = 0; l < S.nlevels; ++l) {
    int lo = S.lvl_sn_ptr[l], hi = S.lvl_sn_ptr[l + 1];
    if (hi == lo) continue;
    int64_t maxf2 = 0;
    int maxw = 1;
    for (int k = lo; k < hi; ++k) {
      int s = S.lvl_sn[k];
      int64_t f = (S.sn_start[s + 1] - S.sn_start[s]) + (S.rptr[s + 1] - S.rptr[s]);
      maxf2 = std::max(maxf2, f * f);
      maxw = std::max(maxw, S.sn_start[s + 1] - S.sn_start[s]);
    }
    int gy = (int)std::min<int64_t>(4096, (maxf2 + 4095) / 4096);
    k_mf_zero<<<dim3(hi - lo, gy), 256, 0, c->stream>>>(P, lo, hi);
    c->stats.kernel_launches += 2;
    int slo = S.lvl_slot_ptr[l], shi = S.lvl_slot_ptr[l + 1];
    if (shi > slo) k_mf_assemble<<<(shi - slo + 255) / 256, 256, 0, c->stream>>>(P, slo, shi, c->G_val);
    {
      // children of this level's supernodes, all ranks in one launch
      const int g0 = l * S.ea_maxrank, g1 = g0 + S.ea_maxrank;
      if (S.ea_ptr[g1] > S.ea_ptr[g0]) {
        int64_t maxf = 1;
        for (int k = lo; k < hi; ++k) {
          int s = S.lvl_sn[k];
          if (S.ch_ptr[s + 1] > S.ch_ptr[s])
            maxf = std::max<int64_t>(maxf, (S.sn_start[s + 1] - S.sn_start[s]) +
                                               (S.rptr[s + 1] - S.rptr[s]));
        }
        int ey = (int)std::min<int64_t>(maxf, 64);
        k_mf_extend_add_level<<<dim3(hi - lo, ey), 128, 0, c->stream>>>(P, lo);
        c->stats.kernel_launches++;
      }
    }
    size_t smd = 2 * (size_t)maxw * maxw * sizeof(double);
    k_mf_diag<<<hi - lo, 128, smd, c->stream>>>(P, lo, c->d_status);
    int plo = S.ptask_ptr[l], phi = S.ptask_ptr[l + 1];
    if (phi > plo) {
      size_t smp = (2 * (size_t)maxw * maxw + 128 * (size_t)(maxw + 1)) * sizeof(double);
      k_mf_panel<<<phi - plo, 256, smp, c->stream>>>(P, plo);
      c->stats.kernel_launches++;
    }
    int tlo = S.tile_ptr[l], thi = S.tile_ptr[l + 1];
    if (thi > tlo) {
      k_mf_schur<<<thi - tlo, 256, 2 * 64 * 65 * sizeof(double), c->stream>>>(P, tlo);
      c->stats.kernel_launches++;
    }
  }
  return cudaGetLastError();
}

cudaError_t factor_kernel_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_mf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * 64 * 64 * 8);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_mf_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (2 * 64 * 64 + 128 * 65) * 8);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_mf_schur, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              2 * 64 * 65 * 8);
}

}  // namespace ers
