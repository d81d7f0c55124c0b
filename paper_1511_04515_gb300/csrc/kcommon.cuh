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

// Grid barrier for a cooperative (co-resident) launch with a deterministic reduction of
// NV per-block partial values: every block writes part[v * gridDim.x + blockIdx.x]; the
// last block to arrive sums them in block order into out[v] and releases the others.
// bar[0] = arrival count, bar[1] = generation.  Bounded: gives up with ST_TIMEOUT.
template <int NV>
__device__ void grid_reduce(const double (&local)[NV], double* part, double* out,
                            unsigned* bar, unsigned* status, double* sh) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) part[v * gridDim.x + blockIdx.x] = local[v];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned gen = ld_acquire_u(bar + 1);
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    s_last = arrived == gridDim.x - 1;
    if (!s_last) {
      int it = 0;
      while (ld_acquire_u(bar + 1) == gen) {
        __nanosleep(40);
        if (++it > SPIN_LIMIT) { atomicOr(status, ST_TIMEOUT); break; }
      }
    }
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int v = 0; v < NV; ++v) {
      double acc = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        acc += __ldcg(part + v * gridDim.x + b);
      acc = block_sum(acc, sh);
      if (threadIdx.x == 0) out[v] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    }
  }
  __syncthreads();
  __threadfence();
}

}  // namespace ers
