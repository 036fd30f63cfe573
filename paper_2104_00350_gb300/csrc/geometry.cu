// Geometry precompute of the hybrid IB / phase-field method (Sec. 4.1), FP64 on the device.
//
// This translation unit is compiled with -fmad=false: the subgrid-point coordinates,
// the march along the normal and the interpolation-point positions decide integer
// outcomes (counts, ghost flags, averaging cells), so each product and sum is rounded
// on its own, in the order written.
#include <cmath>

#include "ibpf_internal.h"
#include "weights.cuh"

namespace ibpf {
namespace {

__device__ __forceinline__ double wall_height(const WallDev& w, double x) {
  if (w.kind == IB_PF_WALL_SINUSOID) return w.p0 + w.p1 * sin(w.w * x);
  return w.p0;
}

// MASK: the cell-centre fractions interpolated bilinearly at (x, y); centres (i + 1/2) h,
// periodic in x, the first and last centre rows continued beyond them
__device__ __forceinline__ double mask_alpha(const WallDev& w, double x, double y) {
  const double fx = x / w.mh - 0.5, fy = y / w.mh - 0.5;
  const double fx0 = floor(fx), fy0 = floor(fy);
  const double tx = fx - fx0, ty = fy - fy0;
  int i0 = (int)fx0 % w.mnx;
  if (i0 < 0) i0 += w.mnx;
  const int i1 = (i0 + 1) % w.mnx;
  const int j0 = min(max((int)fy0, 0), w.mny - 1), j1 = min(max((int)fy0 + 1, 0), w.mny - 1);
  const double* r0 = w.mask + (size_t)j0 * w.mnx;
  const double* r1 = w.mask + (size_t)j1 * w.mnx;
  const double a = (1.0 - tx) * r0[i0] + tx * r0[i1];
  const double b = (1.0 - tx) * r1[i0] + tx * r1[i1];
  return (1.0 - ty) * a + ty * b;
}

// Sec. 4.1.1: "inside or outside the solid wall"
__device__ __forceinline__ bool is_solid(const WallDev& w, double x, double y) {
  if (w.kind == IB_PF_WALL_NONE) return false;
  if (w.kind == IB_PF_WALL_MASK) return mask_alpha(w, x, y) < 0.5;
  return y < wall_height(w, x);
}

// Volume fractions of the three staggered control-volume families (Sec. 4.1.1):
// kind 0 cells (lower-left corner (i h, j h)), kind 1 x1-faces ((i - 1/2) h, j h),
// kind 2 x2-faces (i h, (j - 1/2) h).  alpha = (fluid subgrid points) / 100^2 over the
// points (x0 + (a + 1/2) h/100, y0 + (b + 1/2) h/100).  A volume whose first subpoint row
// lies at or above the highest wall height of its subpoint columns is all fluid; one whose
// last row lies below the lowest is all solid; the rest are counted point by point.
__global__ void k_alpha(WallDev w, int nx, int rows, int kind, double h, double hs,
                        double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= rows) return;
  double x0 = (kind == 1) ? ((double)i - 0.5) * h : (double)i * h;
  double y0 = (kind == 2) ? ((double)j - 0.5) * h : (double)j * h;
  if (w.kind == IB_PF_WALL_NONE) {
    out[(size_t)j * nx + i] = 1.0;
    return;
  }
  double ywmin = INFINITY, ywmax = -INFINITY;
  for (int a = 0; a < kNsub; ++a) {
    double yw = wall_height(w, x0 + ((double)a + 0.5) * hs);
    ywmin = fmin(ywmin, yw);
    ywmax = fmax(ywmax, yw);
  }
  double yfirst = y0 + 0.5 * hs;
  double ylast = y0 + ((double)(kNsub - 1) + 0.5) * hs;
  double alpha;
  if (yfirst >= ywmax) {
    alpha = 1.0;
  } else if (ylast < ywmin) {
    alpha = 0.0;
  } else {
    int count = 0;
    for (int a = 0; a < kNsub; ++a) {
      double yw = wall_height(w, x0 + ((double)a + 0.5) * hs);
      for (int b = 0; b < kNsub; ++b) {
        double y = y0 + ((double)b + 0.5) * hs;
        count += (y < yw) ? 0 : 1;
      }
    }
    alpha = (double)count / (double)(kNsub * kNsub);
  }
  out[(size_t)j * nx + i] = alpha;
}

__global__ void k_solid_centres(WallDev w, int nx, int ny, double h, int* __restrict__ solidc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  solidc[(size_t)j * nx + i] = is_solid(w, ((double)i + 0.5) * h, ((double)j + 0.5) * h) ? 1 : 0;
}

// Ghost points (Sec. 4.1.2): solid cell centres with a fluid centre among the four face
// neighbours (periodic in x1; no neighbour beyond the x2 walls).  Also flags the faces
// re-interpolated after the velocity ghost fill: alpha_face < 1 and a ghost on one side.
__global__ void k_flags(int nx, int ny, const int* __restrict__ solidc,
                        const double* __restrict__ alpha_u, const double* __restrict__ alpha_v,
                        int* __restrict__ gflag, int* __restrict__ fuflag,
                        int* __restrict__ fvflag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  auto ghost = [&](int ii, int jj) -> bool {
    ii = (ii + nx) % nx;
    if (!solidc[(size_t)jj * nx + ii]) return false;
    bool f = !solidc[(size_t)jj * nx + (ii + 1) % nx] || !solidc[(size_t)jj * nx + (ii + nx - 1) % nx];
    if (jj + 1 < ny) f = f || !solidc[(size_t)(jj + 1) * nx + ii];
    if (jj > 0) f = f || !solidc[(size_t)(jj - 1) * nx + ii];
    return f;
  };
  bool g = ghost(i, j);
  size_t c = (size_t)j * nx + i;
  gflag[c] = g ? 1 : 0;
  fuflag[c] = (alpha_u[c] < 1.0 && (g || ghost(i - 1, j))) ? 1 : 0;
  fvflag[c] = (j >= 1 && alpha_v[c] < 1.0 && (g || ghost(i, j - 1))) ? 1 : 0;
}

// Order-preserving compaction of flag[0..n) into idx (one block, 1024 threads).
__global__ void k_compact(const int* __restrict__ flag, int n, int* __restrict__ idx,
                          int* __restrict__ count) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    int k = base + threadIdx.x;
    int f = (k < n) ? flag[k] : 0;
    int x = f;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;
    }
    __syncthreads();
    int incl = x + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (f) idx[carry + incl - 1] = k;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = carry;
}

__global__ void k_cmap(int n, const int* __restrict__ solidc, int* __restrict__ cmap) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) cmap[c] = solidc[c] ? kCellSolid : kCellFluid;
}

__global__ void k_cmap_ghosts(int ng, const int* __restrict__ gcell, int* __restrict__ cmap) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < ng) cmap[gcell[g]] = g;
}

struct GhostArgs {
  WallDev w;
  int nx, ny;
  double h, ds, d1, d2;
  const double* alpha_c;
  const int* cmap;
  const int* gcell;
  double* nrm;
  double* dn;
  double* gamma;
  int* ap1;
  double* w1;
  int* ap2;
  double* w2;
  int* n_fallback;
  int* n_fail;
  int weights;     // ib_pf_weights
};

__device__ __forceinline__ double alpha_at(const GhostArgs& A, int i, int j) {
  j = j < 0 ? 0 : (j >= A.ny ? A.ny - 1 : j);   // mirror rows at the x2 walls
  i = ((i % A.nx) + A.nx) % A.nx;
  return A.alpha_c[(size_t)j * A.nx + i];
}

// corner (i+1/2, j+1/2) gradient of alpha, Eq. NormalVectors_part1
__device__ __forceinline__ void corner_grad(const GhostArgs& A, int i, int j, double& mx,
                                            double& my) {
  double a00 = alpha_at(A, i, j), a10 = alpha_at(A, i + 1, j);
  double a01 = alpha_at(A, i, j + 1), a11 = alpha_at(A, i + 1, j + 1);
  mx = (a10 + a11 - a00 - a01) / (2.0 * A.h);
  my = (a01 + a11 - a00 - a10) / (2.0 * A.h);
}

// fluid face neighbour in the order +x2, -x2, +x1, -x1; false if none
__device__ bool first_fluid_neighbour(const GhostArgs& A, int i, int j, int& ci, int& cj,
                                      double& e1, double& e2) {
  const int di[4] = {0, 0, 1, -1}, dj[4] = {1, -1, 0, 0};
  for (int k = 0; k < 4; ++k) {
    int jj = j + dj[k];
    if (jj < 0 || jj >= A.ny) continue;
    int ii = (i + di[k] + A.nx) % A.nx;
    if (A.cmap[(size_t)jj * A.nx + ii] == kCellFluid) {
      ci = ii;
      cj = jj;
      e1 = (double)di[k];
      e2 = (double)dj[k];
      return true;
    }
  }
  return false;
}

// Averaging points of one interpolation point (Eq. weright averaged): the cell holding
// (px, py) and its four face neighbours, in the order (0,0), (+1,0), (-1,0), (0,+1),
// (0,-1); cells outside the x2 range or with a solid centre are skipped; weights
// 1/h_i^2 normalised by their sum; a coincident point takes the whole weight.
__device__ int averaging_points(const GhostArgs& A, double px, double py, int* idx, double* wt) {
  const int di[kNap] = {0, 1, -1, 0, 0}, dj[kNap] = {0, 0, 0, 1, -1};
  int i0 = (int)floor(px / A.h), j0 = (int)floor(py / A.h);
  int n = 0;
  double d2s[kNap];
  int off[kNap][3];
  double rel[kNap][3];
  for (int k = 0; k < kNap; ++k) {
    int ic = i0 + di[k], jc = j0 + dj[k];
    if (jc < 0 || jc >= A.ny) continue;
    int icw = ((ic % A.nx) + A.nx) % A.nx;
    if (A.cmap[(size_t)jc * A.nx + icw] != kCellFluid) continue;
    double dx = ((double)ic + 0.5) * A.h - px;
    double dy = ((double)jc + 0.5) * A.h - py;
    idx[n] = jc * A.nx + icw;
    d2s[n] = dx * dx + dy * dy;
    off[n][0] = di[k];
    off[n][1] = dj[k];
    off[n][2] = 0;
    rel[n][0] = dx / A.h;
    rel[n][1] = dy / A.h;
    rel[n][2] = 0.0;
    ++n;
  }
  if (n == 0) return 0;
  double tiny = (1.0e-12 * A.h) * (1.0e-12 * A.h);
  for (int k = 0; k < n; ++k) {
    if (d2s[k] < tiny) {
      for (int m = 0; m < n; ++m) wt[m] = (m == k) ? 1.0 : 0.0;
      return n;
    }
  }
  double q = 0.0;
  for (int k = 0; k < n; ++k) {
    wt[k] = 1.0 / d2s[k];
    q += wt[k];
  }
  for (int k = 0; k < n; ++k) wt[k] = wt[k] / q;
  if (A.weights == IB_PF_W_LINEAR && n >= 3 && stencil_spans<2>(off, n))
    linear_exact_weights<2>(wt, rel, n);
  return n;
}

// Per ghost: normal (Eqs. NormalVectors_part1/2), intersect point by marching h/100 along
// the normal to the first point outside the solid and bisecting 60 times, gamma = d1/dn,
// IP1 = G + (dn + d1 + d2) n, IP2 = G + (dn + d1 + 2 d2) n, averaging points + weights.
__global__ void k_ghost_weights(GhostArgs A, int ng) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ng) return;
  const int c = A.gcell[g];
  int i = c % A.nx, j = c / A.nx;
  double m1x, m1y, m2x, m2y, m3x, m3y, m4x, m4y;
  corner_grad(A, i, j, m1x, m1y);
  corner_grad(A, i - 1, j, m2x, m2y);
  corner_grad(A, i, j - 1, m3x, m3y);
  corner_grad(A, i - 1, j - 1, m4x, m4y);
  double mx = (((m1x + m2x) + m3x) + m4x) / 4.0;
  double my = (((m1y + m2y) + m3y) + m4y) / 4.0;
  double n1, n2;
  int fci, fcj;
  double e1, e2;
  bool has_nb = first_fluid_neighbour(A, i, j, fci, fcj, e1, e2);
  if (sqrt(mx * mx + my * my) * A.h < 1.0e-12) {
    n1 = e1;
    n2 = e2;
    atomicAdd(A.n_fallback, 1);
  } else {
    double norm = sqrt(mx * mx + my * my + kEps0);
    n1 = mx / norm;
    n2 = my / norm;
  }
  double gx = ((double)i + 0.5) * A.h, gy = ((double)j + 0.5) * A.h;
  int k = 1;
  while (k <= kMarchMax) {
    double t = (double)k * A.ds;
    if (!is_solid(A.w, gx + t * n1, gy + t * n2)) break;
    ++k;
  }
  if (k > kMarchMax || !has_nb) {
    atomicAdd(A.n_fail, 1);
    k = kMarchMax;
  }
  double lo = (double)(k - 1) * A.ds, hi = (double)k * A.ds;
  for (int it = 0; it < kBisect; ++it) {
    double mid = 0.5 * (lo + hi);
    if (is_solid(A.w, gx + mid * n1, gy + mid * n2)) lo = mid; else hi = mid;
  }
  A.nrm[2 * g] = n1;
  A.nrm[2 * g + 1] = n2;
  A.dn[g] = hi;
  A.gamma[g] = A.d1 / hi;
  double s1 = (hi + A.d1) + A.d2;
  double s2 = (hi + A.d1) + 2.0 * A.d2;
  for (int which = 0; which < 2; ++which) {
    double s = which == 0 ? s1 : s2;
    int idx[kNap];
    double wt[kNap];
    int n = averaging_points(A, gx + s * n1, gy + s * n2, idx, wt);
    if (n == 0) {
      idx[0] = has_nb ? fcj * A.nx + fci : c;
      wt[0] = 1.0;
      n = 1;
      atomicAdd(A.n_fallback, 1);
    }
    int* ap = which == 0 ? A.ap1 : A.ap2;
    double* ww = which == 0 ? A.w1 : A.w2;
    for (int a = 0; a < kNap; ++a) {
      ap[(size_t)g * kNap + a] = a < n ? idx[a] : idx[0];
      ww[(size_t)g * kNap + a] = a < n ? wt[a] : 0.0;
    }
  }
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

}  // namespace

#define IBPF_TRY(x)                        \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) {               \
      err = std::string(#x) + ": " + cudaGetErrorString(e_); \
      return e_;                           \
    }                                      \
  } while (0)

cudaError_t geometry_init(Instance& in, cudaStream_t s, std::string& err) {
  const int nx = in.nx, ny = in.ny;
  const size_t ncell = (size_t)nx * ny;
  Tables& t = in.tab;
  IBPF_TRY(dalloc(&t.alpha_c, ncell));
  IBPF_TRY(dalloc(&t.alpha_u, ncell));
  IBPF_TRY(dalloc(&t.alpha_v, ncell + nx));
  IBPF_TRY(dalloc(&t.solidc, ncell));
  IBPF_TRY(dalloc(&t.cmap, ncell));
  dim3 blk(32, 8);
  const double hs = in.h / kNsub;
  if (in.wall.kind == IB_PF_WALL_MASK) {
    // the caller's fractions (validated on the host); the predicate reads alpha_c
    const double* a = in.geom.alpha;
    IBPF_TRY(cudaMemcpyAsync(t.alpha_c, a, sizeof(double) * ncell, cudaMemcpyHostToDevice, s));
    IBPF_TRY(cudaMemcpyAsync(t.alpha_u, a + ncell, sizeof(double) * ncell, cudaMemcpyHostToDevice, s));
    IBPF_TRY(cudaMemcpyAsync(t.alpha_v, a + 2 * ncell, sizeof(double) * (ncell + nx), cudaMemcpyHostToDevice, s));
    IBPF_TRY(cudaStreamSynchronize(s));
    in.wall.mask = t.alpha_c;
    in.wall.mnx = nx;
    in.wall.mny = ny;
    in.wall.mh = in.h;
  } else {
    k_alpha<<<dim3((nx + 31) / 32, (ny + 7) / 8), blk, 0, s>>>(in.wall, nx, ny, 0, in.h, hs, t.alpha_c);
    k_alpha<<<dim3((nx + 31) / 32, (ny + 7) / 8), blk, 0, s>>>(in.wall, nx, ny, 1, in.h, hs, t.alpha_u);
    k_alpha<<<dim3((nx + 31) / 32, (ny + 8) / 8), blk, 0, s>>>(in.wall, nx, ny + 1, 2, in.h, hs, t.alpha_v);
  }
  k_solid_centres<<<dim3((nx + 31) / 32, (ny + 7) / 8), blk, 0, s>>>(in.wall, nx, ny, in.h, t.solidc);
  IBPF_TRY(cudaGetLastError());
  int *gflag = nullptr, *fuflag = nullptr, *fvflag = nullptr, *idx = nullptr, *cnt = nullptr;
  IBPF_TRY(dalloc(&gflag, ncell));
  IBPF_TRY(dalloc(&fuflag, ncell));
  IBPF_TRY(dalloc(&fvflag, ncell));
  IBPF_TRY(dalloc(&idx, ncell));
  IBPF_TRY(dalloc(&cnt, 3));
  k_flags<<<dim3((nx + 31) / 32, (ny + 7) / 8), blk, 0, s>>>(nx, ny, t.solidc, t.alpha_u, t.alpha_v,
                                                             gflag, fuflag, fvflag);
  int counts[3] = {0, 0, 0};
  int* lists[3] = {nullptr, nullptr, nullptr};
  int* flags[3] = {gflag, fuflag, fvflag};
  for (int q = 0; q < 3; ++q) {
    k_compact<<<1, 1024, 0, s>>>(flags[q], (int)ncell, idx, cnt + q);
    IBPF_TRY(cudaGetLastError());
    IBPF_TRY(cudaMemcpyAsync(&counts[q], cnt + q, sizeof(int), cudaMemcpyDeviceToHost, s));
    IBPF_TRY(cudaStreamSynchronize(s));
    IBPF_TRY(dalloc(&lists[q], (size_t)counts[q]));
    if (counts[q] > 0)
      IBPF_TRY(cudaMemcpyAsync(lists[q], idx, sizeof(int) * counts[q], cudaMemcpyDeviceToDevice, s));
  }
  t.ng = counts[0];
  t.gcell = lists[0];
  t.nfu = counts[1];
  t.fu = lists[1];
  t.nfv = counts[2];
  t.fv = lists[2];
  k_cmap<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>((int)ncell, t.solidc, t.cmap);
  if (t.ng > 0) k_cmap_ghosts<<<(t.ng + 255) / 256, 256, 0, s>>>(t.ng, t.gcell, t.cmap);
  IBPF_TRY(cudaGetLastError());
  IBPF_TRY(cudaStreamSynchronize(s));
  cudaFree(gflag);
  cudaFree(fuflag);
  cudaFree(fvflag);
  cudaFree(idx);
  cudaFree(cnt);
  const int ng = t.ng;
  IBPF_TRY(dalloc(&t.nrm, 2 * (size_t)ng));
  IBPF_TRY(dalloc(&t.dn, (size_t)ng));
  IBPF_TRY(dalloc(&t.gamma, (size_t)ng));
  IBPF_TRY(dalloc(&t.ap1, (size_t)ng * kNap));
  IBPF_TRY(dalloc(&t.w1, (size_t)ng * kNap));
  IBPF_TRY(dalloc(&t.ap2, (size_t)ng * kNap));
  IBPF_TRY(dalloc(&t.w2, (size_t)ng * kNap));
  return cudaSuccess;
}

cudaError_t geometry_weights(Instance& in, cudaStream_t s, int* n_fail, std::string& err) {
  Tables& t = in.tab;
  *n_fail = 0;
  if (t.ng == 0) return cudaSuccess;
  int* counters = nullptr;
  IBPF_TRY(dalloc(&counters, 2));
  IBPF_TRY(cudaMemsetAsync(counters, 0, 2 * sizeof(int), s));
  GhostArgs A;
  A.w = in.wall;
  A.nx = in.nx;
  A.ny = in.ny;
  A.h = in.h;
  A.ds = in.h / kMarchDiv;
  A.d1 = in.prm.d1;
  A.d2 = in.prm.d2;
  A.alpha_c = t.alpha_c;
  A.cmap = t.cmap;
  A.gcell = t.gcell;
  A.nrm = t.nrm;
  A.dn = t.dn;
  A.gamma = t.gamma;
  A.ap1 = t.ap1;
  A.w1 = t.w1;
  A.ap2 = t.ap2;
  A.w2 = t.w2;
  A.n_fallback = counters;
  A.n_fail = counters + 1;
  A.weights = in.prm.weights;
  k_ghost_weights<<<(t.ng + 127) / 128, 128, 0, s>>>(A, t.ng);
  IBPF_TRY(cudaGetLastError());
  int h[2] = {0, 0};
  IBPF_TRY(cudaMemcpyAsync(h, counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  IBPF_TRY(cudaStreamSynchronize(s));
  cudaFree(counters);
  t.n_fallback = h[0];
  *n_fail = h[1];
  return cudaSuccess;
}

}  // namespace ibpf
