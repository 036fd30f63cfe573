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
// in the FP32 form): a shuffle tree within each warp, then over the warps' results; written
// as FP64 at the tile's index.  The last tile of an instance to finish adds the partials
// (each thread a fixed strided subset, then the same two-level tree) in FP64.
template <typename T>
__device__ __forceinline__ void warp_pair_sum(T& hi, T& lo) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const T oh = __shfl_down_sync(0xffffffffu, hi, off), ol = __shfl_down_sync(0xffffffffu, lo, off);
    pair_add(hi, lo, oh, ol);
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = v + __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

template <typename T, int NT>
__device__ void tile_mass(T hi, T lo, int tile, int ntiles, double* __restrict__ partial,
                          unsigned* __restrict__ ticket, double* __restrict__ mass) {
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
  constexpr int NW = NT / 32;
  __shared__ T wh[NW];
  __shared__ T wl[NW];
  __shared__ double wd[NW];
  __shared__ bool last;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  warp_pair_sum(hi, lo);
  if (lane == 0) {
    wh[warp] = hi;
    wl[warp] = lo;
  }
  __syncthreads();
  if (warp == 0) {
    hi = lane < NW ? wh[lane] : T(0);
    lo = lane < NW ? wl[lane] : T(0);
    warp_pair_sum(hi, lo);
    if (lane == 0) {
      partial[tile] = (double)hi + (double)lo;
      __threadfence();
      last = (atomicAdd(ticket, 1u) == (unsigned)ntiles - 1u);
    }
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double sacc = 0.0;
    for (int b = tid; b < ntiles; b += NT) sacc += ((volatile double*)partial)[b];
    sacc = warp_sum(sacc);
    if (lane == 0) wd[warp] = sacc;
    __syncthreads();
    if (warp == 0) {
      sacc = warp_sum(lane < NW ? wd[lane] : 0.0);
      if (lane == 0) {
        *mass = sacc;
        *ticket = 0u;
      }
    }
  }
  __syncthreads();
}

}  // namespace ibpf
