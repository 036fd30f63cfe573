// Device helpers shared by the 2D and 3D steps: constants, the property-law clamp and the
// fixed-order FP64 (or compensated FP32) mass reduction of the correction kernels.
#pragma once

#include <cuda_runtime.h>

#include "ibpf_internal.h"

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
// as FP64 at the tile's index.  The partials are then added in FP64 in two levels (groups of
// kMassGroup tiles, then the groups), each by the last block of its level to finish, each
// in a fixed order.
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

// The two-level final sum of tile_mass (kMassGroup tiles per group, ibpf_internal.h): the
// last tile of a group to finish adds the group's partials, the last group to finish adds
// the group sums, so no block adds more than max(kMassGroup, groups) values.  partial holds
// ntiles + groups doubles, ticket 1 + groups counters (all zero between steps).

// FP64 sum of v over the NT threads of a block in a fixed tree (every thread gets it)
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* wd) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  v = warp_sum(v);
  if (lane == 0) wd[warp] = v;
  __syncthreads();
  v = warp_sum(lane < NW ? wd[lane] : 0.0);
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
  const int grp = tile / kMassGroup, ngrp = (ntiles + kMassGroup - 1) / kMassGroup;
  const int b0 = grp * kMassGroup;
  const int gsz = ntiles - b0 < kMassGroup ? ntiles - b0 : kMassGroup;
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
      last = (atomicAdd(ticket + 1 + grp, 1u) == (unsigned)gsz - 1u);
    }
  }
  __syncthreads();
  if (!last) return;   // the same for every thread of the block
  // the last tile of group grp: the group's sum
  __threadfence();
  double sacc = 0.0;
  for (int b = tid; b < gsz; b += NT) sacc += ((volatile double*)partial)[b0 + b];
  sacc = block_sum<NT>(sacc, wd);
  if (tid == 0) {
    partial[ntiles + grp] = sacc;
    ticket[1 + grp] = 0u;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == (unsigned)ngrp - 1u);
  }
  __syncthreads();
  if (!last) return;
  // the last group: the sum of the group sums
  __threadfence();
  sacc = 0.0;
  for (int b = tid; b < ngrp; b += NT) sacc += ((volatile double*)partial)[ntiles + b];
  __syncthreads();   // wd is reused
  sacc = block_sum<NT>(sacc, wd);
  if (tid == 0) {
    *mass = sacc;
    *ticket = 0u;
  }
}

// Quotient by a density-type factor (rho_f, Re rho_f; both O(1) and positive).  FP32 form:
// __fdividef, within 2 ulp, a fraction of the cost of the IEEE quotient; the FP32 error
// budget is set by FP32 storage.  FP64: the IEEE quotient.
template <typename T>
__device__ __forceinline__ T qdiv(T a, T b) {
  if constexpr (sizeof(T) == 4) return __fdividef(a, b);
  else return a / b;
}

// ---- runs of four x-consecutive FP32 cells per thread (one 16-byte word per field and row)
struct V4 {
  float e[4];
};
__device__ __forceinline__ V4 ld4(const float* __restrict__ f, size_t q) {
  const float4 v = *reinterpret_cast<const float4*>(f + q);
  return V4{{v.x, v.y, v.z, v.w}};
}
__device__ __forceinline__ void st4(float* __restrict__ f, size_t q, const V4& v) {
  *reinterpret_cast<float4*>(f + q) = make_float4(v.e[0], v.e[1], v.e[2], v.e[3]);
}
template <typename F>
__device__ __forceinline__ V4 map4(F f) {
  V4 r;
#pragma unroll
  for (int e = 0; e < 4; ++e) r.e[e] = f(e);
  return r;
}

// x neighbours of a run: l = value left of cell 0, r = value right of cell 3.  The runs of
// one row segment sit on W consecutive lanes (lane gl of the group); the neighbours come
// from the adjacent lanes by shuffles, except at the ends of the group or of the row
// (periodic wrap), where get(linear index) supplies them.  Every lane of the warp must call.
struct X2 {
  float l, r;
};
template <int W, typename G>
__device__ __forceinline__ X2 xnb(const V4& v, int gl, bool row_start, bool row_end, size_t xl,
                                  size_t xr, G get) {
  X2 x;
  x.l = __shfl_up_sync(0xffffffffu, v.e[3], 1, W);
  x.r = __shfl_down_sync(0xffffffffu, v.e[0], 1, W);
  if (gl == 0 || row_start) x.l = get(xl);
  if (gl == W - 1 || row_end) x.r = get(xr);
  return x;
}
__device__ __forceinline__ float left(const V4& v, const X2& x, int e) { return e == 0 ? x.l : v.e[e - 1]; }
__device__ __forceinline__ float right(const V4& v, const X2& x, int e) { return e == 3 ? x.r : v.e[e + 1]; }

}  // namespace ibpf
