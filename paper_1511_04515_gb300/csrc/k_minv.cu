// Explicit inverses of the merged solve blocks, after every refactor of G_k.
//
// A merged block is a dense triangle of the factor (a nested-dissection separator cut into
// supernodes at the width cap).  Its inverse is built by recursive block inversion of the
// pieces: for a range of pieces split as [A 0; B C],
//     inv = [A^-1 0; -C^-1 B A^-1  C^-1]         (unit lower L_G)
//     inv = [A^-1 -A^-1 B C^-1; 0 C^-1]          (upper U_G)
// from the pieces' inverted diagonal blocks (the leaves) and off-diagonal panels.  The host
// plan (symbolic.cpp) lists, phase by phase, the copies of B out of the panels, T = B X and
// the off-diagonal block -X T as jobs cut into 64 x 64 output tiles; one launch per phase.
// A GEMM whose square operand is triangular skips the zero half of its inner products.
#include "ers_internal.h"

namespace ers {

struct MinvArgs {
  const MJob* jobs;
  const int32_t* tiles;
  double* arr[7];        // LDi, UDi, Lo, Uo, ML, MU, scratch
};

__global__ void __launch_bounds__(256) k_minv_phase(MinvArgs A, int t0) {
  __shared__ double sm[64 * 65];                  // transpose tile, or the two GEMM slabs
  double (*Ts)[65] = reinterpret_cast<double (*)[65]>(sm);
  double (*As)[65] = reinterpret_cast<double (*)[65]>(sm);
  double (*Bs)[65] = reinterpret_cast<double (*)[65]>(sm + 16 * 65);
  const int t = t0 + blockIdx.x;
  const MJob J = A.jobs[A.tiles[2 * t]];
  const int tij = A.tiles[2 * t + 1];
  const int i0 = (tij >> 16) * 64, j0 = (tij & 0xffff) * 64;
  const int tid = threadIdx.x;
  const double* Ap = A.arr[J.a_arr] + J.a_off;
  double* Cp = A.arr[J.c_arr] + J.c_off;
  if (J.kind == MJOB_COPY) {
    for (int e = tid; e < 64 * 64; e += 256) {
      const int i = e & 63, j = e >> 6;
      if (i0 + i < J.m && j0 + j < J.n)
        Cp[(i0 + i) + (int64_t)(j0 + j) * J.ldc] = J.alpha * Ap[(i0 + i) + (int64_t)(j0 + j) * J.lda];
    }
    return;
  }
  if (J.kind == MJOB_COPYT) {   // C[i + j ldc] = A[j + i lda], through shared memory
    for (int e = tid; e < 64 * 64; e += 256) {
      const int jj = e & 63, ii = e >> 6;      // read along A's columns (jj contiguous)
      Ts[ii][jj] = (i0 + ii < J.m && j0 + jj < J.n) ? Ap[(j0 + jj) + (int64_t)(i0 + ii) * J.lda] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < 64 * 64; e += 256) {
      const int i = e & 63, j = e >> 6;
      if (i0 + i < J.m && j0 + j < J.n) Cp[(i0 + i) + (int64_t)(j0 + j) * J.ldc] = J.alpha * Ts[i][j];
    }
    return;
  }
  // GEMM tile: C[i0.., j0..] = alpha sum_k A[i, k] B[k, j] over the k range its triangular
  // operand leaves nonzero
  const double* Bp = A.arr[J.b_arr] + J.b_off;
  int kb = 0, ke = J.k;
  if (J.tri & MTRI_B_LOWER) kb = max(kb, j0);
  if (J.tri & MTRI_A_UPPER) kb = max(kb, i0);
  if (J.tri & MTRI_A_LOWER) ke = min(ke, i0 + 64);
  if (J.tri & MTRI_B_UPPER) ke = min(ke, j0 + 64);
  const int tx = tid & 15, ty = tid >> 4;        // rows ty + 16a, columns tx + 16b
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      const int i = e & 63, kk = e >> 6;         // A slab: 64 rows x 16 k, rows contiguous
      As[kk][i] = (i0 + i < J.m && k0 + kk < ke) ? Ap[(i0 + i) + (int64_t)(k0 + kk) * J.lda] : 0.0;
      const int kq = e & 15, j = e >> 4;         // B slab: 16 k x 64 columns, k contiguous
      Bs[kq][j] = (j0 + j < J.n && k0 + kq < ke) ? Bp[(k0 + kq) + (int64_t)(j0 + j) * J.ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double ar[4], br[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) ar[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) br[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += ar[a] * br[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < J.m && j < J.n) Cp[i + (int64_t)j * J.ldc] = J.alpha * acc[a][b];
    }
}

cudaError_t minv_upload(ers_ctx* c) {
  const Symbolic& S = c->sym;
  if (S.mjobs.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)&c->d_mjobs, sizeof(MJob) * S.mjobs.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_mjobs, S.mjobs.data(), sizeof(MJob) * S.mjobs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_mtile, sizeof(int32_t) * S.mtile.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_mtile, S.mtile.data(), sizeof(int32_t) * S.mtile.size(), cudaMemcpyHostToDevice);
  return e;
}

// Run the inversion phases on the context's stream (the refactor's fronts are dead by now,
// so the arena serves as the phases' scratch).
cudaError_t launch_minv(ers_ctx* c) {
  const Symbolic& S = c->sym;
  if (S.mjobs.empty()) return cudaSuccess;
  DevicePlan& P = c->plan;
  cudaError_t e = cudaMemsetAsync(P.ML, 0, sizeof(double) * S.m_total, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.MU, 0, sizeof(double) * S.m_total, c->stream);
  if (e != cudaSuccess) return e;
  MinvArgs A{c->d_mjobs, c->d_mtile, {P.LDi, P.UDi, P.Lo, P.Uo, P.ML, P.MU, P.arena}};
  for (size_t q = 0; q + 1 < S.mphase_ptr.size(); ++q) {
    const int t0 = S.mphase_ptr[q], nt = S.mphase_ptr[q + 1] - t0;
    if (nt <= 0) continue;
    k_minv_phase<<<nt, 256, 0, c->stream>>>(A, t0);
    c->stats.kernel_launches++;
  }
  return cudaGetLastError();
}

}  // namespace ers
