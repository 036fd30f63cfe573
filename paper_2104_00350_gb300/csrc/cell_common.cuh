// Device helpers shared by the 2D and 3D steps: constants, the property-law clamp and the
// fixed-order FP64 (or compensated FP32) mass reduction of the correction kernels.
#pragma once

#include <cuda_runtime.h>

namespace ibpf {

constexpr double kKappa = 1.0606601717798212;   // 3 / (2 sqrt 2)

// C clamped to [-1, 1] for the property laws rho(C), mu(C): keeps rho >= rho0 = min(rho_l,
// rho_g), the bound the Dodd-Ferrante split of Eq. PressurePoisson rests on
template <typename T>
__device__ __forceinline__ T clamp1(T c) {
  return c > T(1) ? T(1) : (c < T(-1) ? T(-1) : c);
}

// (hi, lo) += (b_hi, b_lo) without rounding loss in FP32 (TwoSum, then renormalise); plain
// addition in FP64.
template <typename T>
__device__ __forceinline__ void pair_add(T& hi, T& lo, T b_hi, T b_lo) {
  if constexpr (sizeof(T) == 8) {
    hi = hi + (b_hi + b_lo);
  } else {
    const T s = hi + b_hi;
    const T bb = s - hi;
    const T e = (hi - (s - bb)) + (b_hi - bb);
    const T l = (lo + b_lo) + e;
    hi = s + l;
    lo = l - (hi - s);
  }
}

// Block reduction of one tile's sum of C in a fixed tree (FP64, or compensated FP32 pairs
// in the FP32 form), written as FP64 at the tile's index; the last tile of an instance to
// finish adds the partials in index order in FP64.
template <typename T, int NT>
__device__ void tile_mass(T hi, T lo, int tile, int ntiles, double* __restrict__ partial,
                          unsigned* __restrict__ ticket, double* __restrict__ mass) {
  __shared__ T rh[NT];
  __shared__ T rl[NT];
  __shared__ double red[NT];
  __shared__ bool last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  rh[tid] = hi;
  rl[tid] = lo;
  __syncthreads();
  for (int s = nthr / 2; s > 0; s >>= 1) {
    if (tid < s) {
      T a_hi = rh[tid], a_lo = rl[tid];
      pair_add(a_hi, a_lo, rh[tid + s], rl[tid + s]);
      rh[tid] = a_hi;
      rl[tid] = a_lo;
    }
    __syncthreads();
  }
  if (tid == 0) {
    partial[tile] = (double)rh[0] + (double)rl[0];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == (unsigned)ntiles - 1u);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double sacc = 0.0;
    for (int b = tid; b < ntiles; b += nthr) sacc += ((volatile double*)partial)[b];
    red[tid] = sacc;
    __syncthreads();
    for (int q = nthr / 2; q > 0; q >>= 1) {
      if (tid < q) red[tid] += red[tid + q];
      __syncthreads();
    }
    if (tid == 0) {
      *mass = red[0];
      *ticket = 0u;
    }
  }
  __syncthreads();
}

}  // namespace ibpf
