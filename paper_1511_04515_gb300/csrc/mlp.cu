// Learned step-size controller network: MLP 32 -> 64 -> 64 -> 64 -> 2 with ReLU, BF16 weights,
// BF16 tensor-core operands with FP32 accumulation (mma.sync m16n8k16 bf16), FP32 master
// weights and Adam.  (The paper's controller is the plain rule of Alg. 2; the network proposes
// the next step from the history of accepted steps and the error test of Eq. 15 decides.)
//
// One CTA of 4 warps handles 64 samples: forward (each warp its 16 samples), loss gradient,
// backward through the layers, and weight gradients dW_l = dH_l^T H_{l-1} where warp w owns the
// 16 output rows [16w, 16w+16) of every dW (no two warps write one entry: deterministic).  Per-
// CTA partial gradients are summed in block order by a second kernel, then Adam updates the FP32
// master weights and refreshes the BF16 copy.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "ers_internal.h"

namespace ers {

constexpr int NIN = 32, NH = 64, NOUT = 2;
constexpr int SPB = 64;   // samples per CTA
// FP32 parameter vector layout
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN;
constexpr int OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH;
constexpr int OFF_W4 = OFF_B3 + NH, OFF_B4 = OFF_W4 + NOUT * NH;
constexpr int NPARAM = OFF_B4 + NOUT;   // 10562
// BF16 working copy of the weights: W1 (64x32), W2, W3 (64x64), W4 padded to 16 x 64
constexpr int BW1 = 0, BW2 = BW1 + NH * NIN, BW3 = BW2 + NH * NH, BW4 = BW3 + NH * NH;
constexpr int NBW = BW4 + 16 * NH;

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D(16x8) += A(16x16, row) * B(16x8, col); bf16 inputs, fp32 accumulators
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A fragment of a 16x16 tile whose element (r, c) is at M[(r0 + r) * rs + (c0 + c) * cs]
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const __nv_bfloat16* M, int r0, int c0,
                                       int rs, int cs, int lane) {
  int g = lane >> 2, t = lane & 3;
  auto at = [&](int r, int c) { return M[(r0 + r) * rs + (c0 + c) * cs]; };
  a[0] = pack2(at(g, 2 * t), at(g, 2 * t + 1));
  a[1] = pack2(at(g + 8, 2 * t), at(g + 8, 2 * t + 1));
  a[2] = pack2(at(g, 2 * t + 8), at(g, 2 * t + 9));
  a[3] = pack2(at(g + 8, 2 * t + 8), at(g + 8, 2 * t + 9));
}

// B fragment of a 16x8 tile (k x n) whose element (k, n) is at M[(k0 + k) * ks + (n0 + n) * ns]
__device__ __forceinline__ void load_b(uint32_t (&b)[2], const __nv_bfloat16* M, int k0, int n0,
                                       int ks, int ns, int lane) {
  int g = lane >> 2, t = lane & 3;
  auto at = [&](int k, int n) { return M[(k0 + k) * ks + (n0 + n) * ns]; };
  b[0] = pack2(at(2 * t, g), at(2 * t + 1, g));
  b[1] = pack2(at(2 * t + 8, g), at(2 * t + 9, g));
}

struct MlpArgs {
  const __nv_bfloat16* W;   // NBW
  const float* P;           // NPARAM (biases are read from here)
  const float* X;           // n x 32
  const float* T;           // n x 2 (train)
  int n;
  int train;
  float* Y;                 // n x 2 (inference), may be null in training
  float* partial;           // gridDim.x x (NPARAM + 1) (train): gradients and loss
  float inv_n;              // 1 / (samples of the whole minibatch)
};

// Row strides of the shared-memory tiles, padded by 8 bf16 (16 bytes) so that the fragment
// loads of one warp touch 32 distinct banks.
constexpr int LD0 = NIN + 8, LDH = NH + 8, LD4 = 16 + 8;
constexpr int SM_W1 = 0, SM_W2 = SM_W1 + NH * LD0, SM_W3 = SM_W2 + NH * LDH;
constexpr int SM_W4 = SM_W3 + NH * LDH, SM_H0 = SM_W4 + 16 * LDH;
constexpr int SM_H = SM_H0 + 2 * SPB * LD0, SM_D = SM_H + 6 * SPB * LDH;
constexpr int SM_D4 = SM_D + 6 * SPB * LDH, SM_BF16 = SM_D4 + 2 * SPB * LD4;
constexpr size_t MLP_SMEM = SM_BF16 * 2 + (SPB * NOUT + 4) * sizeof(float);

// An activation or delta v is held as the pair (hi, lo) = (bf16(v), bf16(v - hi)), so that it
// keeps about 16 significant bits while every tensor-core operand stays BF16 (the weights are
// BF16 by definition).  A product with a weight takes two MMAs (hi and lo); a product of two
// pairs takes three (the lo x lo term is below FP32 rounding).
struct Pair {
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
};
__device__ __forceinline__ void put(const Pair& P, int idx, float v) {
  __nv_bfloat16 h = __float2bfloat16(v);
  P.hi[idx] = h;
  P.lo[idx] = __float2bfloat16(v - __bfloat162float(h));
}
__device__ __forceinline__ float get(const Pair& P, int idx) {
  return __bfloat162float(P.hi[idx]) + __bfloat162float(P.lo[idx]);
}

// shared memory: weights W1 (64x32), W2, W3 (64x64), W4 (16x64, rows 2..15 zero), and as
// (hi, lo) pairs the activations H0 (64 samples x 32), H1..H3 (64x64), the deltas D1..D3
// (64x64) and the output delta D4 (64 x 16)
__global__ void __launch_bounds__(128) k_mlp(MlpArgs A) {
  extern __shared__ __align__(16) unsigned char mlp_smem[];
  __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(mlp_smem);
  __nv_bfloat16* sW1 = sb + SM_W1;
  __nv_bfloat16* sW2 = sb + SM_W2;
  __nv_bfloat16* sW3 = sb + SM_W3;
  __nv_bfloat16* sW4 = sb + SM_W4;
  const Pair sH0{sb + SM_H0, sb + SM_H0 + SPB * LD0};
  Pair sH[3], sD[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    sH[l] = Pair{sb + SM_H + (2 * l) * SPB * LDH, sb + SM_H + (2 * l + 1) * SPB * LDH};
    sD[l] = Pair{sb + SM_D + (2 * l) * SPB * LDH, sb + SM_D + (2 * l + 1) * SPB * LDH};
  }
  const Pair sD4{sb + SM_D4, sb + SM_D4 + SPB * LD4};
  float* sY = reinterpret_cast<float*>(sb + SM_BF16);
  float* sLoss = sY + SPB * NOUT;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int base = blockIdx.x * SPB;
  for (int e = tid; e < NH * NIN; e += blockDim.x)
    sW1[(e / NIN) * LD0 + e % NIN] = A.W[BW1 + e];
  for (int e = tid; e < NH * NH; e += blockDim.x) {
    sW2[(e / NH) * LDH + e % NH] = A.W[BW2 + e];
    sW3[(e / NH) * LDH + e % NH] = A.W[BW3 + e];
  }
  for (int e = tid; e < 16 * NH; e += blockDim.x) sW4[(e / NH) * LDH + e % NH] = A.W[BW4 + e];
  for (int e = tid; e < SPB * NIN; e += blockDim.x) {
    int s = e / NIN, f = e % NIN;
    float v = (base + s < A.n) ? A.X[(int64_t)(base + s) * NIN + f] : 0.0f;
    put(sH0, s * LD0 + f, v);
  }
  __syncthreads();
  const int g = lane >> 2, t = lane & 3;
  const int r0 = 16 * w;   // this warp's samples
  // ---- forward: H_l = relu(H_{l-1} W_l^T + b_l), output Y = H3 W4^T + b4
  const __nv_bfloat16* Wl[3] = {sW1, sW2, sW3};
  const int Kin[3] = {NIN, NH, NH};
  const int LDin[3] = {LD0, LDH, LDH};
  const int boff[3] = {OFF_B1, OFF_B2, OFF_B3};
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const Pair in = l == 0 ? sH0 : sH[l - 1];
    const int K = Kin[l], ld = LDin[l];
    for (int nt = 0; nt < NH / 8; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      for (int kt = 0; kt < K / 16; ++kt) {
        uint32_t ah[4], al[4], b[2];
        load_b(b, Wl[l], kt * 16, nt * 8, 1, ld, lane);   // W[o][i]: (k=i, n=o)
        load_a(ah, in.hi, r0, kt * 16, ld, 1, lane);
        load_a(al, in.lo, r0, kt * 16, ld, 1, lane);
        mma16816(d, ah, b);
        mma16816(d, al, b);
      }
      int c = nt * 8 + 2 * t;
      float b0 = A.P[boff[l] + c], b1 = A.P[boff[l] + c + 1];
      put(sH[l], (r0 + g) * LDH + c, fmaxf(d[0] + b0, 0.f));
      put(sH[l], (r0 + g) * LDH + c + 1, fmaxf(d[1] + b1, 0.f));
      put(sH[l], (r0 + g + 8) * LDH + c, fmaxf(d[2] + b0, 0.f));
      put(sH[l], (r0 + g + 8) * LDH + c + 1, fmaxf(d[3] + b1, 0.f));
    }
    __syncwarp();
  }
  {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    for (int kt = 0; kt < NH / 16; ++kt) {
      uint32_t ah[4], al[4], b[2];
      load_b(b, sW4, kt * 16, 0, 1, LDH, lane);   // rows 2..15 of W4 are zero
      load_a(ah, sH[2].hi, r0, kt * 16, LDH, 1, lane);
      load_a(al, sH[2].lo, r0, kt * 16, LDH, 1, lane);
      mma16816(d, ah, b);
      mma16816(d, al, b);
    }
    if (t == 0) {   // columns 0 and 1 of the 16 x 8 result
      sY[(r0 + g) * NOUT + 0] = d[0] + A.P[OFF_B4 + 0];
      sY[(r0 + g) * NOUT + 1] = d[1] + A.P[OFF_B4 + 1];
      sY[(r0 + g + 8) * NOUT + 0] = d[2] + A.P[OFF_B4 + 0];
      sY[(r0 + g + 8) * NOUT + 1] = d[3] + A.P[OFF_B4 + 1];
    }
  }
  __syncthreads();
  if (!A.train) {
    for (int e = tid; e < SPB * NOUT; e += blockDim.x) {
      int s = e / NOUT;
      if (base + s < A.n) A.Y[(int64_t)(base + s) * NOUT + e % NOUT] = sY[e];
    }
    return;
  }
  // ---- loss L = (1/n) sum_s sum_o (Y - T)^2, output delta D4 = dL/dY (padded to 16 cols)
  float lsum = 0.f;
  for (int e = tid; e < SPB * 16; e += blockDim.x) {
    int s = e / 16, o = e % 16;
    float dv = 0.f;
    if (o < NOUT && base + s < A.n) {
      float diff = sY[s * NOUT + o] - A.T[(int64_t)(base + s) * NOUT + o];
      lsum += diff * diff;
      dv = 2.f * diff * A.inv_n;
    }
    put(sD4, s * LD4 + o, dv);
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) sLoss[w] = lsum;
  __syncthreads();
  // ---- backward: D_l = (D_{l+1} W_{l+1}) * relu'(H_l), l = 3, 2, 1 (stored in sD[l-1])
  const __nv_bfloat16* Wnext[3] = {sW2, sW3, sW4};
#pragma unroll
  for (int l = 2; l >= 0; --l) {
    const Pair dnext = l == 2 ? sD4 : sD[l + 1];
    const int Kd = l == 2 ? 16 : NH;    // width of D_{l+1}
    const int ldd = l == 2 ? LD4 : LDH;
    for (int nt = 0; nt < NH / 8; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      for (int kt = 0; kt < Kd / 16; ++kt) {
        uint32_t ah[4], al[4], b[2];
        load_b(b, Wnext[l], kt * 16, nt * 8, LDH, 1, lane);   // W_{l+1}[o][i]: (k=o, n=i)
        load_a(ah, dnext.hi, r0, kt * 16, ldd, 1, lane);
        load_a(al, dnext.lo, r0, kt * 16, ldd, 1, lane);
        mma16816(d, ah, b);
        mma16816(d, al, b);
      }
      int c = nt * 8 + 2 * t;
      auto gate = [&](int s, int cc, float v) {
        float hv = __bfloat162float(sH[l].hi[s * LDH + cc]);
        put(sD[l], s * LDH + cc, hv > 0.f ? v : 0.f);
      };
      gate(r0 + g, c, d[0]);
      gate(r0 + g, c + 1, d[1]);
      gate(r0 + g + 8, c, d[2]);
      gate(r0 + g + 8, c + 1, d[3]);
    }
    __syncwarp();
  }
  __syncthreads();
  // ---- weight gradients dW_l = D_l^T H_{l-1} (64 x K_in), warp w owns rows [16w, 16w+16)
  float* part = A.partial + (int64_t)blockIdx.x * (NPARAM + 1);
  const int woff[3] = {OFF_W1, OFF_W2, OFF_W3};
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const Pair hin = l == 0 ? sH0 : sH[l - 1];
    const int K = Kin[l], ld = LDin[l];
    for (int nt = 0; nt < K / 8; ++nt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      for (int kt = 0; kt < SPB / 16; ++kt) {   // reduction over the CTA's samples
        uint32_t ah[4], al[4], bh[2], bl[2];
        load_a(ah, sD[l].hi, r0, kt * 16, 1, LDH, lane);   // (o, s) at s*LDH + o
        load_a(al, sD[l].lo, r0, kt * 16, 1, LDH, lane);
        load_b(bh, hin.hi, kt * 16, nt * 8, ld, 1, lane);  // (s, i) at s*ld + i
        load_b(bl, hin.lo, kt * 16, nt * 8, ld, 1, lane);
        mma16816(d, ah, bh);
        mma16816(d, ah, bl);
        mma16816(d, al, bh);
      }
      int o = r0 + g, i = nt * 8 + 2 * t;
      part[woff[l] + o * K + i] = d[0];
      part[woff[l] + o * K + i + 1] = d[1];
      part[woff[l] + (o + 8) * K + i] = d[2];
      part[woff[l] + (o + 8) * K + i + 1] = d[3];
    }
  }
  // output layer dW4 (2 x 64) and all biases: plain FP32 sums over the CTA's samples
  for (int e = tid; e < NOUT * NH; e += blockDim.x) {
    int o = e / NH, i = e % NH;
    float acc = 0.f;
    for (int s = 0; s < SPB; ++s) acc += get(sD4, s * LD4 + o) * get(sH[2], s * LDH + i);
    part[OFF_W4 + e] = acc;
  }
  for (int e = tid; e < 3 * NH + NOUT; e += blockDim.x) {
    float acc = 0.f;
    if (e < 3 * NH) {
      int l = e / NH, o = e % NH;
      const Pair D = l == 0 ? sD[0] : (l == 1 ? sD[1] : sD[2]);
      for (int s = 0; s < SPB; ++s) acc += get(D, s * LDH + o);
      part[boff[l] + o] = acc;
    } else {
      int o = e - 3 * NH;
      for (int s = 0; s < SPB; ++s) acc += get(sD4, s * LD4 + o);
      part[OFF_B4 + o] = acc;
    }
  }
  if (tid == 0) part[NPARAM] = sLoss[0] + sLoss[1] + sLoss[2] + sLoss[3];
}

// grad[p] = sum over blocks (fixed order) of partial[b][p]; p = NPARAM is the loss sum
__global__ void k_mlp_reduce(const float* partial, int nblocks, float* grad) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NPARAM) return;
  float acc = 0.f;
  for (int b = 0; b < nblocks; ++b) acc += partial[(int64_t)b * (NPARAM + 1) + p];
  grad[p] = acc;
}

// Adam on the FP32 master weights, then the BF16 working copy
__global__ void k_mlp_adam(float* P, float* m, float* v, const float* grad, float lr, float b1,
                           float b2, float eps, float c1, float c2, __nv_bfloat16* W) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  float gr = grad[p];
  float mm = b1 * m[p] + (1.f - b1) * gr;
  float vv = b2 * v[p] + (1.f - b2) * gr * gr;
  m[p] = mm;
  v[p] = vv;
  float w = P[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  P[p] = w;
  // BF16 copy
  __nv_bfloat16 bw = __float2bfloat16(w);
  if (p < OFF_B1) W[BW1 + p] = bw;
  else if (p >= OFF_W2 && p < OFF_B2) W[BW2 + (p - OFF_W2)] = bw;
  else if (p >= OFF_W3 && p < OFF_B3) W[BW3 + (p - OFF_W3)] = bw;
  else if (p >= OFF_W4 && p < OFF_B4) W[BW4 + (p - OFF_W4)] = bw;
}

__global__ void k_mlp_to_bf16(const float* P, __nv_bfloat16* W) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NBW) return;
  float v = 0.f;
  if (e < BW2) v = P[OFF_W1 + e];
  else if (e < BW3) v = P[OFF_W2 + (e - BW2)];
  else if (e < BW4) v = P[OFF_W3 + (e - BW3)];
  else {
    int q = e - BW4;   // padded 16 x 64
    if (q < NOUT * NH) v = P[OFF_W4 + q];
  }
  W[e] = __float2bfloat16(v);
}

}  // namespace ers

// ---------------------------------------------------------------------------------------
// C ABI of the network
// ---------------------------------------------------------------------------------------
struct ers_mlp {
  std::string err;
  float* P = nullptr;        // NPARAM fp32 master
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;     // NPARAM + 1
  __nv_bfloat16* W = nullptr;
  float* partial = nullptr;
  int partial_blocks = 0;
  float *dX = nullptr, *dT = nullptr, *dY = nullptr;
  int cap = 0;
  int64_t adam_t = 0;
  cudaStream_t stream = nullptr;
};

using namespace ers;

namespace {

ers_status mfail(ers_mlp* M, const std::string& msg) {
  if (M) M->err = msg;
  return ERS_ERR_CUDA;
}
#define MCU(call)                                                             \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) return mfail(M, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

ers_status ensure_cap(ers_mlp* M, int n) {
  int blocks = (n + SPB - 1) / SPB;
  if (n > M->cap) {
    cudaFree(M->dX);
    cudaFree(M->dT);
    cudaFree(M->dY);
    MCU(cudaMalloc(&M->dX, sizeof(float) * (size_t)n * NIN));
    MCU(cudaMalloc(&M->dT, sizeof(float) * (size_t)n * NOUT));
    MCU(cudaMalloc(&M->dY, sizeof(float) * (size_t)n * NOUT));
    M->cap = n;
  }
  if (blocks > M->partial_blocks) {
    cudaFree(M->partial);
    MCU(cudaMalloc(&M->partial, sizeof(float) * (size_t)blocks * (NPARAM + 1)));
    M->partial_blocks = blocks;
  }
  return ERS_OK;
}

}  // namespace

extern "C" {

int32_t ers_mlp_nparam(void) { return NPARAM; }

ers_status ers_mlp_create(ers_mlp** out, uint64_t seed) {
  if (!out) return ERS_ERR_INVALID;
  ers_mlp* M = new ers_mlp();
  *out = M;
  MCU(cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking));
  MCU(cudaFuncSetAttribute(k_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM));
  MCU(cudaMalloc(&M->P, sizeof(float) * NPARAM));
  MCU(cudaMalloc(&M->m, sizeof(float) * NPARAM));
  MCU(cudaMalloc(&M->v, sizeof(float) * NPARAM));
  MCU(cudaMalloc(&M->grad, sizeof(float) * (NPARAM + 1)));
  MCU(cudaMalloc(&M->W, sizeof(__nv_bfloat16) * NBW));
  MCU(cudaMemset(M->m, 0, sizeof(float) * NPARAM));
  MCU(cudaMemset(M->v, 0, sizeof(float) * NPARAM));
  // He initialisation of the weights, zero biases (host generator, seeded)
  std::vector<float> P(NPARAM, 0.f);
  std::mt19937_64 rng(seed);
  auto init = [&](int off, int fan_in, int count) {
    std::normal_distribution<float> nd(0.f, std::sqrt(2.f / fan_in));
    for (int k = 0; k < count; ++k) P[off + k] = nd(rng);
  };
  init(OFF_W1, NIN, NH * NIN);
  init(OFF_W2, NH, NH * NH);
  init(OFF_W3, NH, NH * NH);
  init(OFF_W4, NH, NOUT * NH);
  return ers_mlp_set_params(M, P.data());
}

ers_status ers_mlp_set_params(ers_mlp* M, const float* params) {
  if (!M || !params) return ERS_ERR_INVALID;
  MCU(cudaMemcpyAsync(M->P, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, M->stream));
  k_mlp_to_bf16<<<(NBW + 255) / 256, 256, 0, M->stream>>>(M->P, M->W);
  MCU(cudaGetLastError());
  MCU(cudaStreamSynchronize(M->stream));
  return ERS_OK;
}

ers_status ers_mlp_get_params(const ers_mlp* MM, float* params) {
  ers_mlp* M = const_cast<ers_mlp*>(MM);
  if (!M || !params) return ERS_ERR_INVALID;
  MCU(cudaMemcpyAsync(params, M->P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, M->stream));
  MCU(cudaStreamSynchronize(M->stream));
  return ERS_OK;
}

ers_status ers_mlp_forward_dev(ers_mlp* M, const float* X_dev, int32_t n, float* Y_dev,
                               void* stream) {
  if (!M || n < 0) return ERS_ERR_INVALID;
  if (n == 0) return ERS_OK;
  MlpArgs A{M->W, M->P, X_dev, nullptr, n, 0, Y_dev, nullptr, 0.f};
  k_mlp<<<(n + SPB - 1) / SPB, 128, MLP_SMEM, stream ? (cudaStream_t)stream : M->stream>>>(A);
  MCU(cudaGetLastError());
  return ERS_OK;
}

ers_status ers_mlp_forward(ers_mlp* M, const float* X, int32_t n, float* Y) {
  if (!M || (n > 0 && (!X || !Y))) return ERS_ERR_INVALID;
  if (n == 0) return ERS_OK;
  ers_status st = ensure_cap(M, n);
  if (st != ERS_OK) return st;
  MCU(cudaMemcpyAsync(M->dX, X, sizeof(float) * (size_t)n * NIN, cudaMemcpyHostToDevice, M->stream));
  st = ers_mlp_forward_dev(M, M->dX, n, M->dY, M->stream);
  if (st != ERS_OK) return st;
  MCU(cudaMemcpyAsync(Y, M->dY, sizeof(float) * (size_t)n * NOUT, cudaMemcpyDeviceToHost, M->stream));
  MCU(cudaStreamSynchronize(M->stream));
  return ERS_OK;
}

static ers_status mlp_grad_dev(ers_mlp* M, const float* dX, const float* dT, int n) {
  int blocks = (n + SPB - 1) / SPB;
  MlpArgs A{M->W, M->P, dX, dT, n, 1, nullptr, M->partial, 1.f / (float)n};
  k_mlp<<<blocks, 128, MLP_SMEM, M->stream>>>(A);
  k_mlp_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, M->stream>>>(M->partial, blocks, M->grad);
  MCU(cudaGetLastError());
  return ERS_OK;
}

static ers_status mlp_adam_dev(ers_mlp* M, const float* dX, const float* dT, int n, float lr) {
  ers_status st = mlp_grad_dev(M, dX, dT, n);
  if (st != ERS_OK) return st;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  ++M->adam_t;
  float c1 = 1.f - std::pow(b1, (float)M->adam_t), c2 = 1.f - std::pow(b2, (float)M->adam_t);
  k_mlp_adam<<<(NPARAM + 255) / 256, 256, 0, M->stream>>>(M->P, M->m, M->v, M->grad, lr, b1, b2,
                                                           eps, c1, c2, M->W);
  MCU(cudaGetLastError());
  return ERS_OK;
}

ers_status ers_mlp_grad(ers_mlp* M, const float* X, const float* T, int32_t n, float* grad,
                        float* loss) {
  if (!M || n <= 0 || !X || !T) return ERS_ERR_INVALID;
  ers_status st = ensure_cap(M, n);
  if (st != ERS_OK) return st;
  MCU(cudaMemcpyAsync(M->dX, X, sizeof(float) * (size_t)n * NIN, cudaMemcpyHostToDevice, M->stream));
  MCU(cudaMemcpyAsync(M->dT, T, sizeof(float) * (size_t)n * NOUT, cudaMemcpyHostToDevice, M->stream));
  st = mlp_grad_dev(M, M->dX, M->dT, n);
  if (st != ERS_OK) return st;
  std::vector<float> g(NPARAM + 1);
  MCU(cudaMemcpyAsync(g.data(), M->grad, sizeof(float) * (NPARAM + 1), cudaMemcpyDeviceToHost, M->stream));
  MCU(cudaStreamSynchronize(M->stream));
  if (grad) std::memcpy(grad, g.data(), sizeof(float) * NPARAM);
  if (loss) *loss = g[NPARAM] / (float)n;
  return ERS_OK;
}

ers_status ers_mlp_adam_step(ers_mlp* M, const float* X, const float* T, int32_t n, float lr,
                            float* loss) {
  if (!M || n <= 0 || !X || !T || !(lr > 0.f)) return ERS_ERR_INVALID;
  ers_status st = ensure_cap(M, n);
  if (st != ERS_OK) return st;
  MCU(cudaMemcpyAsync(M->dX, X, sizeof(float) * (size_t)n * NIN, cudaMemcpyHostToDevice, M->stream));
  MCU(cudaMemcpyAsync(M->dT, T, sizeof(float) * (size_t)n * NOUT, cudaMemcpyHostToDevice, M->stream));
  st = mlp_adam_dev(M, M->dX, M->dT, n, lr);
  if (st != ERS_OK) return st;
  float lsum = 0.f;
  MCU(cudaMemcpyAsync(&lsum, M->grad + NPARAM, sizeof(float), cudaMemcpyDeviceToHost, M->stream));
  MCU(cudaStreamSynchronize(M->stream));
  if (loss) *loss = lsum / (float)n;
  return ERS_OK;
}

ers_status ers_mlp_train(ers_mlp* M, const float* X, const float* T, int32_t n, int32_t epochs,
                         int32_t batch, float lr, uint64_t seed, float* final_loss) {
  if (!M || n <= 0 || !X || !T || epochs < 1 || batch < 1 || !(lr > 0.f)) return ERS_ERR_INVALID;
  batch = std::min(batch, n);
  ers_status st = ensure_cap(M, n);
  if (st != ERS_OK) return st;
  // each epoch uploads the dataset in a seeded random order and takes one Adam step per
  // minibatch of `batch` consecutive samples
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::mt19937_64 rng(seed);
  std::vector<float> xs((size_t)n * NIN), ts((size_t)n * NOUT);
  float last = 0.f;
  int last_nb = batch;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    for (int k = 0; k < n; ++k) {
      std::memcpy(&xs[(size_t)k * NIN], &X[(size_t)order[k] * NIN], sizeof(float) * NIN);
      std::memcpy(&ts[(size_t)k * NOUT], &T[(size_t)order[k] * NOUT], sizeof(float) * NOUT);
    }
    MCU(cudaMemcpyAsync(M->dX, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice, M->stream));
    MCU(cudaMemcpyAsync(M->dT, ts.data(), sizeof(float) * ts.size(), cudaMemcpyHostToDevice, M->stream));
    for (int b0 = 0; b0 < n; b0 += batch) {
      last_nb = std::min(batch, n - b0);
      st = mlp_adam_dev(M, M->dX + (size_t)b0 * NIN, M->dT + (size_t)b0 * NOUT, last_nb, lr);
      if (st != ERS_OK) return st;
    }
    // the host buffers are refilled next epoch: wait for the uploads and steps to finish
    MCU(cudaMemcpyAsync(&last, M->grad + NPARAM, sizeof(float), cudaMemcpyDeviceToHost, M->stream));
    MCU(cudaStreamSynchronize(M->stream));
  }
  if (final_loss) *final_loss = last / (float)last_nb;
  return ERS_OK;
}

const char* ers_mlp_last_error(const ers_mlp* M) { return M ? M->err.c_str() : "null"; }

void ers_mlp_destroy(ers_mlp* M) {
  if (!M) return;
  for (void* p : {(void*)M->P, (void*)M->m, (void*)M->v, (void*)M->grad, (void*)M->W,
                  (void*)M->partial, (void*)M->dX, (void*)M->dT, (void*)M->dY})
    if (p) cudaFree(p);
  if (M->stream) cudaStreamDestroy(M->stream);
  delete M;
}

}  // extern "C"
