// Small device helpers shared by the kernels: memory-ordering primitives, bounded waits,
// warp / block reductions and a bounded grid barrier with a deterministic reduction.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ers_internal.h"

namespace ers {

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(int32_t* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spin until *p >= target; gives up after SPIN_LIMIT polls (sets ST_TIMEOUT) or as soon as
// another waiter has timed out.  Returns false on give-up.  Called by one thread.
__device__ __forceinline__ bool wait_geq(const int32_t* p, int target, unsigned* status) {
  if (ld_acquire(p) >= target) return true;
  for (int it = 0; it < SPIN_LIMIT; ++it) {
    __nanosleep(it < 64 ? 20 : 200);
    if (ld_acquire(p) >= target) return true;
    if ((it & 255) == 255 && (ld_acquire_u(status) & ST_TIMEOUT)) return false;
  }
  atomicOr(status, ST_TIMEOUT);
  return false;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block sum (deterministic: fixed tree).  sh must hold blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  double r = 0.0;
  if (wid == 0) {
    r = lane < nw ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  v = warp_max(v);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  double r = 0.0;
  if (wid == 0) {
    r = lane < nw ? sh[lane] : 0.0;
    r = warp_max(r);
  }
  __syncthreads();
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// Sums NV per-thread values over the block; every thread receives the NV totals.  Each warp
// reduces with the xor butterfly (all lanes end with the same bits), then every thread adds
// the warp totals in warp order: the result is fixed by the data, not by timing.
// sh: NV * blockDim.x / 32 doubles.
template <int NV>
__device__ __forceinline__ void block_sum_n(double (&v)[NV], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * nw + wid] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double a = 0.0;
    for (int q = 0; q < nw; ++q) a += sh[k * nw + q];
    v[k] = a;
  }
  __syncthreads();
}

__device__ __forceinline__ void red_release_add_u(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spin until *p >= target (one thread); bounded like wait_geq, with short first polls since
// the grid reductions that use it wait for microseconds.
__device__ __forceinline__ void wait_geq_u(const unsigned* p, unsigned target, unsigned* status) {
  if (ld_acquire_u(p) >= target) return;
  for (int it = 0; it < SPIN_LIMIT; ++it) {
    if (it >= 16) __nanosleep(it < 256 ? 32 : 256);
    if (ld_acquire_u(p) >= target) return;
    if ((it & 255) == 255 && (ld_acquire_u(status) & ST_TIMEOUT)) return;
  }
  atomicOr(status, ST_TIMEOUT);
}

// Grid-wide reductions and barriers of a cooperative (co-resident) launch.  bar[0] counts the
// blocks' arrivals over the whole launch (the r-th reduction completes when it reaches
// (r + 1) * gridDim.x) and bar[1] their exits; both are zero at launch and reset by the last
// block to leave (grid_exit).  A block publishes its partials and arrives with one release
// add; after the acquire every block reads all partials and sums them in block order, so all
// blocks hold the same total with no second hand-off.  The partial slots alternate between
// two halves by round parity: a block can only write round r + 2's partials after every block
// has arrived at round r + 1, i.e. finished reading round r's.  Bounded: ST_TIMEOUT.
constexpr int GRID_RED_NV = 2 * MAX_RHS;   // most values reduced at once
struct GridRed {
  double* part;        // 2 * GRID_RED_NV * gridDim.x doubles
  unsigned* bar;
  unsigned* status;
  unsigned round;
};

// v: per-thread values in, grid totals out (all threads of all blocks).
// sh: NV * (blockDim.x / 32) doubles.
template <int NV>
__device__ __forceinline__ void grid_sum_n(double (&v)[NV], GridRed& g, double* sh) {
  static_assert(NV <= GRID_RED_NV, "too many values");
  block_sum_n<NV>(v, sh);
  const unsigned G = gridDim.x;
  if (G == 1) return;
  double* slot = g.part + (size_t)(g.round & 1u) * (GRID_RED_NV * G);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) slot[k * G + blockIdx.x] = v[k];
    red_release_add_u(g.bar, 1u);
    wait_geq_u(g.bar, (g.round + 1u) * G, g.status);
  }
  g.round++;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (wid < NV) {               // one warp per value: the block-order sum in lane-strided parts
    double a = 0.0;
    for (unsigned b = lane; b < G; b += 32) a += __ldcg(slot + wid * G + b);
    a = warp_sum(a);
    if (lane == 0) sh[wid] = a;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = sh[k];
  __syncthreads();
}

// Every block's writes before the call are visible to every block after it.
__device__ __forceinline__ void grid_sync(GridRed& g) {
  __syncthreads();
  const unsigned G = gridDim.x;
  if (G == 1) return;
  if (threadIdx.x == 0) {
    red_release_add_u(g.bar, 1u);
    wait_geq_u(g.bar, (g.round + 1u) * G, g.status);
  }
  g.round++;
  __syncthreads();
}

// Last call of a kernel that used grid_sum_n / grid_sync: the last block out resets the
// counters for the next launch (every other block is past its last wait by then).
__device__ __forceinline__ void grid_exit(GridRed& g) {
  if (gridDim.x == 1 || threadIdx.x != 0) return;
  if (atomicAdd(g.bar + 1, 1u) == gridDim.x - 1) {
    atomicExch(g.bar, 0u);
    atomicExch(g.bar + 1, 0u);
  }
}

}  // namespace ers
