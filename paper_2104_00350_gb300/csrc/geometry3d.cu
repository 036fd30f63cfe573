// Geometry precompute of the hybrid IB / phase-field method in 3D (Sec. 4.1), FP64 on the
// device: volume fractions of the four control-volume families by subgrid counting, cell
// classes, the ghost list, normals from corner gradients of alpha, intersect / mirror /
// interpolation points, the 7-point inverse-distance stencils W1/W2 and the list of faces
// re-interpolated after the velocity ghost fill.
//
// Compiled with -fmad=false, like the 2D geometry: subgrid coordinates, sphere distances,
// the march along the normal and the interpolation-point positions decide integer outcomes,
// so every product and sum is rounded on its own, in the order written.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "ibpf_internal.h"
#include "weights.cuh"

namespace ibpf {
namespace {

// nearest periodic image of a coordinate difference: shifted by -L above L/2, +L below -L/2
__device__ __forceinline__ double wrapd(double d, double L) {
  if (d > 0.5 * L) d = d - L;
  if (d < -0.5 * L) d = d + L;
  return d;
}

__device__ __forceinline__ bool in_sphere(const WallDev& w, const Sph& s, double x, double y,
                                          double z) {
  const double dx = wrapd(x - s.x, w.lx), dy = wrapd(y - s.y, w.ly), dz = z - s.z;
  return ((dx * dx + dy * dy) + dz * dz) < s.r * s.r;
}

__device__ __forceinline__ int bin_axis(double x, double L, double bs, int nb, bool periodic) {
  if (periodic) x = x - floor(x / L) * L;
  int b = (int)floor(x / bs);
  return b < 0 ? 0 : (b >= nb ? nb - 1 : b);
}

__device__ __forceinline__ int bin_of(const WallDev& w, double x, double y, double z) {
  const SphereSet& s = w.ss;
  const int bx = bin_axis(x, w.lx, s.bs[0], s.nb[0], true);
  const int by = bin_axis(y, w.ly, s.bs[1], s.nb[1], true);
  const int bz = bin_axis(z, w.lz, s.bs[2], s.nb[2], false);
  return (bz * s.nb[1] + by) * s.nb[0] + bx;
}

// MASK: the cell-centre fractions interpolated trilinearly at (x, y, z); centres (i + 1/2) h,
// periodic in x and y, the first and last centre planes continued beyond them
__device__ double mask_alpha3(const WallDev& w, double x, double y, double z) {
  const double fx = x / w.mh - 0.5, fy = y / w.mh - 0.5, fz = z / w.mh - 0.5;
  const double fx0 = floor(fx), fy0 = floor(fy), fz0 = floor(fz);
  const double tx = fx - fx0, ty = fy - fy0, tz = fz - fz0;
  int i0 = (int)fx0 % w.mnx, j0 = (int)fy0 % w.mny;
  if (i0 < 0) i0 += w.mnx;
  if (j0 < 0) j0 += w.mny;
  const int i1 = (i0 + 1) % w.mnx, j1 = (j0 + 1) % w.mny;
  const int k0 = min(max((int)fz0, 0), w.mnz - 1), k1 = min(max((int)fz0 + 1, 0), w.mnz - 1);
  const size_t nxy = (size_t)w.mnx * w.mny;
  const double* p0 = w.mask + (size_t)k0 * nxy;
  const double* p1 = w.mask + (size_t)k1 * nxy;
  auto plane = [&](const double* p) {
    const double a = (1.0 - tx) * p[(size_t)j0 * w.mnx + i0] + tx * p[(size_t)j0 * w.mnx + i1];
    const double b = (1.0 - tx) * p[(size_t)j1 * w.mnx + i0] + tx * p[(size_t)j1 * w.mnx + i1];
    return (1.0 - ty) * a + ty * b;
  };
  return (1.0 - tz) * plane(p0) + tz * plane(p1);
}

// Sec. 4.1.1: is (x, y, z) inside the solid?
__device__ bool is_solid3(const WallDev& w, double x, double y, double z) {
  if (w.kind == IB_PF_WALL_NONE) return false;
  if (w.kind == IB_PF_WALL_FLAT) return z < w.p0;
  if (w.kind == IB_PF_WALL_MASK) return mask_alpha3(w, x, y, z) < 0.5;
  const int b = bin_of(w, x, y, z);
  for (int q = w.ss.bstart[b]; q < w.ss.bstart[b + 1]; ++q)
    if (in_sphere(w, w.ss.sph[w.ss.blist[q]], x, y, z)) return true;
  return false;
}

// Fluid fraction of the control volumes of one family: volume (k, j, i) has its lower corner
// at ((i + sx) h, (j + sy) h, (k + sz) h); alpha = fluid points / 16^3 over the points
// (x0 + (a + 1/2) h/16, ...).  A sphere whose nearest point of the volume lies at or beyond
// its radius holds none of the points; a sphere holding all 8 corners holds all of them
// (convexity); only the remaining spheres are tested point by point.
constexpr int kBand = 8;
__global__ void k_alpha3(WallDev w, int nx, int ny, int nplanes, double sx, double sy,
                         double sz, double h, double* __restrict__ out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t total = (size_t)nx * ny * nplanes;
  if (idx >= total) return;
  const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((size_t)nx * ny));
  const double x0 = ((double)i + sx) * h, y0 = ((double)j + sy) * h, z0 = ((double)k + sz) * h;
  const double hs = h / (double)kNsub3;
  double alpha = 1.0;
  if (w.kind == IB_PF_WALL_FLAT) {
    int cnt = 0;
    for (int a = 0; a < kNsub3; ++a) cnt += (z0 + ((double)a + 0.5) * hs >= w.p0) ? 1 : 0;
    alpha = (double)(cnt * kNsub3 * kNsub3) / (double)(kNsub3 * kNsub3 * kNsub3);
  } else if (w.kind != IB_PF_WALL_NONE) {
    const double hh = 0.5 * h;
    const double xc = x0 + hh, yc = y0 + hh, zc = z0 + hh;
    const int b = bin_of(w, xc, yc, zc);
    int band[kBand];
    int nband = 0;
    bool overflow = false, full = false;
    for (int q = w.ss.bstart[b]; q < w.ss.bstart[b + 1]; ++q) {
      const Sph s = w.ss.sph[w.ss.blist[q]];
      const double ax = fabs(wrapd(xc - s.x, w.lx)), ay = fabs(wrapd(yc - s.y, w.ly));
      const double az = fabs(zc - s.z);
      const double nx_ = fmax(ax - hh, 0.0), ny_ = fmax(ay - hh, 0.0), nz_ = fmax(az - hh, 0.0);
      if ((nx_ * nx_ + ny_ * ny_) + nz_ * nz_ >= s.r * s.r) continue;    // no point inside
      const double fx = ax + hh, fy = ay + hh, fz = az + hh;
      if ((fx * fx + fy * fy) + fz * fz < s.r * s.r) { full = true; break; }   // all inside
      if (nband < kBand) band[nband++] = w.ss.blist[q];
      else overflow = true;
    }
    if (full) {
      alpha = 0.0;
    } else if (nband > 0) {
      int cnt = 0;
      for (int c = 0; c < kNsub3; ++c) {
        const double z = z0 + ((double)c + 0.5) * hs;
        for (int bb = 0; bb < kNsub3; ++bb) {
          const double y = y0 + ((double)bb + 0.5) * hs;
          for (int a = 0; a < kNsub3; ++a) {
            const double x = x0 + ((double)a + 0.5) * hs;
            bool in = false;
            if (!overflow) {
              for (int q = 0; q < nband && !in; ++q) in = in_sphere(w, w.ss.sph[band[q]], x, y, z);
            } else {
              in = is_solid3(w, x, y, z);
            }
            cnt += in ? 0 : 1;
          }
        }
      }
      alpha = (double)cnt / (double)(kNsub3 * kNsub3 * kNsub3);
    }
  }
  out[idx] = alpha;
}

__global__ void k_solid_centres3(WallDev w, int nx, int ny, int nz, double h,
                                 int* __restrict__ solidc) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)nx * ny * nz) return;
  const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / ((size_t)nx * ny));
  solidc[idx] =
      is_solid3(w, ((double)i + 0.5) * h, ((double)j + 0.5) * h, ((double)k + 0.5) * h) ? 1 : 0;
}

// ghost flag: solid centre with a fluid centre among the 6 face neighbours (periodic x, y;
// no neighbour beyond the z walls)
__global__ void k_ghost_flags3(int nx, int ny, int nz, const int* __restrict__ solidc,
                               uint8_t* __restrict__ flag) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nxy = (size_t)nx * ny;
  if (idx >= nxy * nz) return;
  const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / nxy);
  uint8_t g = 0;
  if (solidc[idx]) {
    const size_t r = idx - i;                 // start of row (k, j)
    const size_t p = idx - (size_t)j * nx;    // cell (k, 0, i)
    bool fl = !solidc[r + (i + 1) % nx] || !solidc[r + (i + nx - 1) % nx] ||
              !solidc[p + (size_t)((j + 1) % ny) * nx] || !solidc[p + (size_t)((j + ny - 1) % ny) * nx];
    if (k + 1 < nz) fl = fl || !solidc[idx + nxy];
    if (k > 0) fl = fl || !solidc[idx - nxy];
    g = fl ? 1 : 0;
  }
  flag[idx] = g;
}

// faces re-interpolated after the velocity ghost fill: alpha_face < 1 and a ghost cell on
// one side; axis 0 x-faces (cells i-1, i), 1 y-faces (j-1, j), 2 z-faces k = 1..nz-1
__global__ void k_face_flags3(int nx, int ny, int nz, int axis, const uint8_t* __restrict__ ghost,
                              const double* __restrict__ alpha, uint8_t* __restrict__ flag) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t nxy = (size_t)nx * ny;
  const size_t total = axis == 2 ? nxy * (nz + 1) : nxy * nz;
  if (idx >= total) return;
  const int i = (int)(idx % nx), j = (int)((idx / nx) % ny), k = (int)(idx / nxy);
  uint8_t f = 0;
  if (axis == 0) {
    f = (alpha[idx] < 1.0 && (ghost[idx] || ghost[idx - i + (i + nx - 1) % nx])) ? 1 : 0;
  } else if (axis == 1) {
    const size_t below = idx - (size_t)j * nx + (size_t)((j + ny - 1) % ny) * nx;
    f = (alpha[idx] < 1.0 && (ghost[idx] || ghost[below])) ? 1 : 0;
  } else if (k >= 1 && k <= nz - 1) {
    f = (alpha[idx] < 1.0 && (ghost[idx] || ghost[idx - nxy])) ? 1 : 0;
  }
  flag[idx] = f;
}

// ordered stream compaction of a byte flag array: block counts, a host prefix, then each
// block writes the indices of its flagged elements in order
constexpr int kCompactThreads = 256, kCompactItems = 16;
constexpr int kCompactSpan = kCompactThreads * kCompactItems;

__global__ void k_flag_count(const uint8_t* __restrict__ flag, size_t n, int* __restrict__ cnt) {
  __shared__ int red[kCompactThreads];
  const size_t base = (size_t)blockIdx.x * kCompactSpan + (size_t)threadIdx.x * kCompactItems;
  int c = 0;
  for (int q = 0; q < kCompactItems; ++q)
    if (base + q < n) c += flag[base + q];
  red[threadIdx.x] = c;
  __syncthreads();
  for (int s = kCompactThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[blockIdx.x] = red[0];
}

__global__ void k_flag_scatter(const uint8_t* __restrict__ flag, size_t n,
                               const int* __restrict__ offs, int* __restrict__ out) {
  __shared__ int scan[kCompactThreads];
  const size_t base = (size_t)blockIdx.x * kCompactSpan + (size_t)threadIdx.x * kCompactItems;
  int c = 0;
  for (int q = 0; q < kCompactItems; ++q)
    if (base + q < n) c += flag[base + q];
  scan[threadIdx.x] = c;
  __syncthreads();
  for (int s = 1; s < kCompactThreads; s <<= 1) {   // inclusive Hillis-Steele scan
    const int v = (int)threadIdx.x >= s ? scan[threadIdx.x - s] : 0;
    __syncthreads();
    scan[threadIdx.x] += v;
    __syncthreads();
  }
  int pos = offs[blockIdx.x] + scan[threadIdx.x] - c;
  for (int q = 0; q < kCompactItems; ++q)
    if (base + q < n && flag[base + q]) out[pos++] = (int)(base + q);
}

__global__ void k_cmap3(size_t n, const int* __restrict__ solidc, int* __restrict__ cmap) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) cmap[idx] = solidc[idx] ? kCellSolid : kCellFluid;
}

__global__ void k_cmap_ghosts3(int ng, const int* __restrict__ gcell, int* __restrict__ cmap) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < ng) cmap[gcell[g]] = g;
}

struct Ghost3Args {
  WallDev w;
  int nx, ny, nz, ng;
  double h, d1, d2;
  const int* gcell;
  const int* cmap;
  const double* alpha_c;
  double* nrm;     // ng x 3
  double* dn;
  double* gamma;
  int* ap1;        // ng x 7
  double* w1;
  int* ap2;
  double* w2;
  int* n_fail;     // ghosts without an intersect point within 10 h
  int* n_fallback;
  int weights;     // ib_pf_weights
};

__device__ __forceinline__ double alpha_at3(const Ghost3Args& a, int i, int j, int k) {
  k = k < 0 ? 0 : (k >= a.nz ? a.nz - 1 : k);     // mirror planes at the z walls
  i = ((i % a.nx) + a.nx) % a.nx;
  j = ((j % a.ny) + a.ny) % a.ny;
  return a.alpha_c[((size_t)k * a.ny + j) * a.nx + i];
}

__device__ __forceinline__ bool fluid_at(const Ghost3Args& a, int i, int j, int k) {
  if (k < 0 || k >= a.nz) return false;
  i = ((i % a.nx) + a.nx) % a.nx;
  j = ((j % a.ny) + a.ny) % a.ny;
  return a.cmap[((size_t)k * a.ny + j) * a.nx + i] == kCellFluid;
}

// first fluid face neighbour in the order +z, -z, +x, -x, +y, -y; returns its direction
__device__ bool first_fluid3(const Ghost3Args& a, int i, int j, int k, int& di, int& dj, int& dk) {
  const int dirs[6][3] = {{0, 0, 1}, {0, 0, -1}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}};
  for (int q = 0; q < 6; ++q) {
    if (fluid_at(a, i + dirs[q][0], j + dirs[q][1], k + dirs[q][2])) {
      di = dirs[q][0];
      dj = dirs[q][1];
      dk = dirs[q][2];
      return true;
    }
  }
  return false;
}

// the cell holding p and its 6 face neighbours, fluid centres only, inverse-squared-distance
// weights normalised; a coincident point takes the whole weight.  Returns the count.
__device__ int averaging3(const Ghost3Args& a, double px, double py, double pz, int* ap,
                          double* wt) {
  const double h = a.h;
  const int i0 = (int)floor(px / h), j0 = (int)floor(py / h), k0 = (int)floor(pz / h);
  const int off[7][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  double d2s[kNap3];
  int koff[kNap3][3];
  double rel[kNap3][3];
  int n = 0;
  for (int q = 0; q < kNap3; ++q) {
    const int ic = i0 + off[q][0], jc = j0 + off[q][1], kc = k0 + off[q][2];
    if (!fluid_at(a, ic, jc, kc)) continue;
    const double dx = ((double)ic + 0.5) * h - px;
    const double dy = ((double)jc + 0.5) * h - py;
    const double dz = ((double)kc + 0.5) * h - pz;
    const int im = ((ic % a.nx) + a.nx) % a.nx, jm = ((jc % a.ny) + a.ny) % a.ny;
    ap[n] = (kc * a.ny + jm) * a.nx + im;
    d2s[n] = (dx * dx + dy * dy) + dz * dz;
    for (int k = 0; k < 3; ++k) koff[n][k] = off[q][k];
    rel[n][0] = dx / h;
    rel[n][1] = dy / h;
    rel[n][2] = dz / h;
    ++n;
  }
  if (n == 0) return 0;
  const double tiny = (1.0e-12 * h) * (1.0e-12 * h);
  for (int q = 0; q < n; ++q) {
    if (d2s[q] < tiny) {
      for (int r = 0; r < n; ++r) wt[r] = r == q ? 1.0 : 0.0;
      return n;
    }
  }
  double s = 0.0;
  for (int q = 0; q < n; ++q) {
    wt[q] = 1.0 / d2s[q];
    s = s + wt[q];
  }
  for (int q = 0; q < n; ++q) wt[q] = wt[q] / s;
  if (a.weights == IB_PF_W_LINEAR && n >= 4 && stencil_spans<3>(koff, n))
    linear_exact_weights<3>(wt, rel, n);
  return n;
}

// Sec. 4.1.2 for one ghost: normal (corner gradients of alpha, Eqs. NormalVectors in 3D),
// intersect point (march h/100 along n, then 60 bisections), mirror and interpolation
// points IP1 = M + d2 n, IP2 = M + 2 d2 n, and their averaging stencils.
__global__ void k_ghost_weights3(Ghost3Args a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.ng) return;
  const int c = a.gcell[g];
  const int i = c % a.nx, j = (c / a.nx) % a.ny, k = c / (a.nx * a.ny);
  const double h = a.h;
  // corner (ci+1/2, cj+1/2, ck+1/2): differences of the two 2 x 2 faces of its 8 cells / 4h
  double m[3] = {0.0, 0.0, 0.0};
  for (int dk = -1; dk <= 0; ++dk)
    for (int dj = -1; dj <= 0; ++dj)
      for (int di = -1; di <= 0; ++di) {
        const int ci = i + di, cj = j + dj, ck = k + dk;
        double v[2][2][2];   // v[dk][dj][di]
        for (int ek = 0; ek < 2; ++ek)
          for (int ej = 0; ej < 2; ++ej)
            for (int ei = 0; ei < 2; ++ei) v[ek][ej][ei] = alpha_at3(a, ci + ei, cj + ej, ck + ek);
        const double mx = ((v[0][0][1] + v[0][1][1]) + (v[1][0][1] + v[1][1][1]) -
                           ((v[0][0][0] + v[0][1][0]) + (v[1][0][0] + v[1][1][0]))) / (4.0 * h);
        const double my = ((v[0][1][0] + v[0][1][1]) + (v[1][1][0] + v[1][1][1]) -
                           ((v[0][0][0] + v[0][0][1]) + (v[1][0][0] + v[1][0][1]))) / (4.0 * h);
        const double mz = ((v[1][0][0] + v[1][0][1]) + (v[1][1][0] + v[1][1][1]) -
                           ((v[0][0][0] + v[0][0][1]) + (v[0][1][0] + v[0][1][1]))) / (4.0 * h);
        m[0] = m[0] + mx;
        m[1] = m[1] + my;
        m[2] = m[2] + mz;
      }
  for (int q = 0; q < 3; ++q) m[q] = m[q] / 8.0;
  const double mag2 = (m[0] * m[0] + m[1] * m[1]) + m[2] * m[2];
  double n1, n2, n3;
  if (sqrt(mag2) * h < 1.0e-12) {
    int di = 0, dj = 0, dk = 0;
    first_fluid3(a, i, j, k, di, dj, dk);
    n1 = (double)di;
    n2 = (double)dj;
    n3 = (double)dk;
    atomicAdd(a.n_fallback, 1);
  } else {
    const double nrm = sqrt(mag2 + kEps0);
    n1 = m[0] / nrm;
    n2 = m[1] / nrm;
    n3 = m[2] / nrm;
  }
  a.nrm[3 * (size_t)g] = n1;
  a.nrm[3 * (size_t)g + 1] = n2;
  a.nrm[3 * (size_t)g + 2] = n3;
  const double gx = ((double)i + 0.5) * h, gy = ((double)j + 0.5) * h, gz = ((double)k + 0.5) * h;
  const double ds = h / (double)kMarchDiv;
  int q = 1;
  while (q <= kMarchMax) {
    const double t = (double)q * ds;
    if (!is_solid3(a.w, gx + t * n1, gy + t * n2, gz + t * n3)) break;
    ++q;
  }
  if (q > kMarchMax) {
    atomicAdd(a.n_fail, 1);
    a.dn[g] = h;
    a.gamma[g] = a.d1 / h;
    for (int r = 0; r < kNap3; ++r) {
      a.ap1[(size_t)g * kNap3 + r] = c;
      a.ap2[(size_t)g * kNap3 + r] = c;
      a.w1[(size_t)g * kNap3 + r] = 0.0;
      a.w2[(size_t)g * kNap3 + r] = 0.0;
    }
    return;
  }
  double lo = (double)(q - 1) * ds, hi = (double)q * ds;
  for (int b = 0; b < kBisect; ++b) {
    const double mid = 0.5 * (lo + hi);
    if (is_solid3(a.w, gx + mid * n1, gy + mid * n2, gz + mid * n3)) lo = mid;
    else hi = mid;
  }
  a.dn[g] = hi;
  a.gamma[g] = a.d1 / hi;
  const double s1 = (hi + a.d1) + a.d2;
  const double s2 = (hi + a.d1) + 2.0 * a.d2;
  for (int which = 0; which < 2; ++which) {
    const double s = which == 0 ? s1 : s2;
    int* ap = which == 0 ? a.ap1 : a.ap2;
    double* wt = which == 0 ? a.w1 : a.w2;
    int idx[kNap3];
    double w[kNap3];
    int n = averaging3(a, gx + s * n1, gy + s * n2, gz + s * n3, idx, w);
    if (n == 0) {
      int di = 0, dj = 0, dk = 0;
      first_fluid3(a, i, j, k, di, dj, dk);
      const int im = ((i + di) % a.nx + a.nx) % a.nx, jm = ((j + dj) % a.ny + a.ny) % a.ny;
      idx[0] = ((k + dk) * a.ny + jm) * a.nx + im;
      w[0] = 1.0;
      n = 1;
      atomicAdd(a.n_fallback, 1);
    }
    for (int r = 0; r < kNap3; ++r) {
      ap[(size_t)g * kNap3 + r] = r < n ? idx[r] : idx[0];
      wt[(size_t)g * kNap3 + r] = r < n ? w[r] : 0.0;
    }
  }
}

template <typename T>
cudaError_t dalloc3(T** p, size_t n) {
  return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

// ordered indices of the flagged elements of flag[0..n) into a new device array
cudaError_t compact3(const uint8_t* flag, size_t n, int** out, int* count, cudaStream_t s) {
  const size_t nb = (n + kCompactSpan - 1) / kCompactSpan;
  int* cnt = nullptr;
  cudaError_t e = dalloc3(&cnt, nb);
  if (e != cudaSuccess) return e;
  k_flag_count<<<(unsigned)nb, kCompactThreads, 0, s>>>(flag, n, cnt);
  std::vector<int> h(nb);
  e = cudaMemcpyAsync(h.data(), cnt, sizeof(int) * nb, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cudaFree(cnt); return e; }
  long long tot = 0;
  for (size_t b = 0; b < nb; ++b) {
    const int c = h[b];
    h[b] = (int)tot;
    tot += c;
  }
  *count = (int)tot;
  e = dalloc3(out, (size_t)tot);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cnt, h.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && tot > 0) k_flag_scatter<<<(unsigned)nb, kCompactThreads, 0, s>>>(flag, n, cnt, *out);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(cnt);
  return e;
}

unsigned blocks_for(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

#define IBPF_TRY3(x)                                         \
  do {                                                       \
    cudaError_t e_ = (x);                                    \
    if (e_ != cudaSuccess) {                                 \
      err = std::string(#x) + ": " + cudaGetErrorString(e_); \
      return e_;                                             \
    }                                                        \
  } while (0)

cudaError_t geometry3_init(Instance& in, const double* h_spheres, int n_spheres, cudaStream_t s,
                           std::string& err) {
  const int nx = in.nx, ny = in.ny, nz = in.nz;
  const size_t nxy = (size_t)nx * ny, ncell = nxy * nz, nwf = ncell + nxy;
  const double h = in.h;
  Tables& t = in.tab;
  t.nap = kNap3;
  WallDev& w = in.wall;
  w.lx = in.lx;
  w.ly = in.ly;
  w.lz = in.lz;
  // sphere set and its bins (one bin per 8 cells along each axis, at most 64 per axis)
  if (w.kind == IB_PF_WALL_SPHERE || w.kind == IB_PF_WALL_SPHERES) {
    std::vector<Sph> sph;
    if (w.kind == IB_PF_WALL_SPHERE) {
      sph.push_back(Sph{in.geom.p[0], in.geom.p[1], in.geom.p[2], in.geom.p[3]});
    } else {
      for (int q = 0; q < n_spheres; ++q)
        sph.push_back(Sph{h_spheres[4 * q], h_spheres[4 * q + 1], h_spheres[4 * q + 2],
                          h_spheres[4 * q + 3]});
    }
    const int ncells[3] = {nx, ny, nz};
    const double L[3] = {in.lx, in.ly, in.lz};
    int nb[3];
    double bs[3];
    for (int a = 0; a < 3; ++a) {
      nb[a] = std::max(1, std::min(64, ncells[a] / 8));
      bs[a] = L[a] / nb[a];
    }
    const size_t nbins = (size_t)nb[0] * nb[1] * nb[2];
    std::vector<std::vector<int>> lists(nbins);
    for (size_t q = 0; q < sph.size(); ++q) {
      const double c[3] = {sph[q].x, sph[q].y, sph[q].z};
      const double ext = sph[q].r + h;   // bounding box grown by one cell
      int lo[3], hi[3];
      for (int a = 0; a < 3; ++a) {
        lo[a] = (int)std::floor((c[a] - ext) / bs[a]);
        hi[a] = (int)std::floor((c[a] + ext) / bs[a]);
        if (a < 2) {
          if (hi[a] - lo[a] + 1 >= nb[a]) { lo[a] = 0; hi[a] = nb[a] - 1; }
        } else {
          lo[a] = std::max(0, std::min(nb[a] - 1, lo[a]));
          hi[a] = std::max(0, std::min(nb[a] - 1, hi[a]));
        }
      }
      for (int bz = lo[2]; bz <= hi[2]; ++bz)
        for (int by = lo[1]; by <= hi[1]; ++by)
          for (int bx = lo[0]; bx <= hi[0]; ++bx) {
            const int ix = ((bx % nb[0]) + nb[0]) % nb[0], iy = ((by % nb[1]) + nb[1]) % nb[1];
            lists[((size_t)bz * nb[1] + iy) * nb[0] + ix].push_back((int)q);
          }
    }
    std::vector<int> start(nbins + 1, 0), flat;
    for (size_t b = 0; b < nbins; ++b) {
      start[b + 1] = start[b] + (int)lists[b].size();
      flat.insert(flat.end(), lists[b].begin(), lists[b].end());
    }
    IBPF_TRY3(dalloc3(&in.sph, sph.size()));
    IBPF_TRY3(dalloc3(&in.bstart, nbins + 1));
    IBPF_TRY3(dalloc3(&in.blist, flat.size()));
    IBPF_TRY3(cudaMemcpy(in.sph, sph.data(), sizeof(Sph) * sph.size(), cudaMemcpyHostToDevice));
    IBPF_TRY3(cudaMemcpy(in.bstart, start.data(), sizeof(int) * (nbins + 1), cudaMemcpyHostToDevice));
    if (!flat.empty())
      IBPF_TRY3(cudaMemcpy(in.blist, flat.data(), sizeof(int) * flat.size(), cudaMemcpyHostToDevice));
    w.ss.sph = in.sph;
    w.ss.bstart = in.bstart;
    w.ss.blist = in.blist;
    for (int a = 0; a < 3; ++a) {
      w.ss.nb[a] = nb[a];
      w.ss.bs[a] = bs[a];
    }
  }
  IBPF_TRY3(dalloc3(&t.alpha_c, ncell));
  IBPF_TRY3(dalloc3(&t.alpha_u, ncell));
  IBPF_TRY3(dalloc3(&t.alpha_v, ncell));
  IBPF_TRY3(dalloc3(&t.alpha_w, nwf));
  IBPF_TRY3(dalloc3(&t.solidc, ncell));
  IBPF_TRY3(dalloc3(&t.cmap, ncell));
  const int T = 128;
  if (w.kind == IB_PF_WALL_MASK) {
    // the caller's fractions (validated on the host); the predicate reads alpha_c
    const double* a = in.geom.alpha;
    IBPF_TRY3(cudaMemcpyAsync(t.alpha_c, a, sizeof(double) * ncell, cudaMemcpyHostToDevice, s));
    IBPF_TRY3(cudaMemcpyAsync(t.alpha_u, a + ncell, sizeof(double) * ncell, cudaMemcpyHostToDevice, s));
    IBPF_TRY3(cudaMemcpyAsync(t.alpha_v, a + 2 * ncell, sizeof(double) * ncell, cudaMemcpyHostToDevice, s));
    IBPF_TRY3(cudaMemcpyAsync(t.alpha_w, a + 3 * ncell, sizeof(double) * nwf, cudaMemcpyHostToDevice, s));
    IBPF_TRY3(cudaStreamSynchronize(s));
    w.mask = t.alpha_c;
    w.mnx = nx;
    w.mny = ny;
    w.mnz = nz;
    w.mh = h;
  } else {
    k_alpha3<<<blocks_for(ncell, T), T, 0, s>>>(w, nx, ny, nz, 0.0, 0.0, 0.0, h, t.alpha_c);
    k_alpha3<<<blocks_for(ncell, T), T, 0, s>>>(w, nx, ny, nz, -0.5, 0.0, 0.0, h, t.alpha_u);
    k_alpha3<<<blocks_for(ncell, T), T, 0, s>>>(w, nx, ny, nz, 0.0, -0.5, 0.0, h, t.alpha_v);
    k_alpha3<<<blocks_for(nwf, T), T, 0, s>>>(w, nx, ny, nz + 1, 0.0, 0.0, -0.5, h, t.alpha_w);
  }
  k_solid_centres3<<<blocks_for(ncell, 256), 256, 0, s>>>(w, nx, ny, nz, h, t.solidc);
  IBPF_TRY3(cudaGetLastError());
  uint8_t *gflag = nullptr, *fflag = nullptr;
  IBPF_TRY3(dalloc3(&gflag, ncell));
  IBPF_TRY3(dalloc3(&fflag, nwf));
  k_ghost_flags3<<<blocks_for(ncell, 256), 256, 0, s>>>(nx, ny, nz, t.solidc, gflag);
  IBPF_TRY3(cudaGetLastError());
  IBPF_TRY3(compact3(gflag, ncell, &t.gcell, &t.ng, s));
  k_cmap3<<<blocks_for(ncell, 256), 256, 0, s>>>(ncell, t.solidc, t.cmap);
  if (t.ng > 0) k_cmap_ghosts3<<<blocks_for(t.ng, 256), 256, 0, s>>>(t.ng, t.gcell, t.cmap);
  IBPF_TRY3(cudaGetLastError());
  const double* alphas[3] = {t.alpha_u, t.alpha_v, t.alpha_w};
  int* counts[3] = {&t.nfu, &t.nfv, &t.nfw};
  int** lists3[3] = {&t.fu, &t.fv, &t.fw};
  for (int a = 0; a < 3; ++a) {
    const size_t n = a == 2 ? nwf : ncell;
    k_face_flags3<<<blocks_for(n, 256), 256, 0, s>>>(nx, ny, nz, a, gflag, alphas[a], fflag);
    IBPF_TRY3(cudaGetLastError());
    IBPF_TRY3(compact3(fflag, n, lists3[a], counts[a], s));
  }
  IBPF_TRY3(cudaStreamSynchronize(s));
  cudaFree(gflag);
  cudaFree(fflag);
  const size_t ng = (size_t)t.ng;
  IBPF_TRY3(dalloc3(&t.nrm, 3 * ng));
  IBPF_TRY3(dalloc3(&t.dn, ng));
  IBPF_TRY3(dalloc3(&t.gamma, ng));
  IBPF_TRY3(dalloc3(&t.ap1, ng * kNap3));
  IBPF_TRY3(dalloc3(&t.w1, ng * kNap3));
  IBPF_TRY3(dalloc3(&t.ap2, ng * kNap3));
  IBPF_TRY3(dalloc3(&t.w2, ng * kNap3));
  return cudaSuccess;
}

cudaError_t geometry3_weights(Instance& in, cudaStream_t s, int* n_fail, std::string& err) {
  Tables& t = in.tab;
  *n_fail = 0;
  if (t.ng == 0) return cudaSuccess;
  int* counters = nullptr;
  IBPF_TRY3(dalloc3(&counters, 2));
  IBPF_TRY3(cudaMemsetAsync(counters, 0, 2 * sizeof(int), s));
  Ghost3Args A;
  A.w = in.wall;
  A.nx = in.nx;
  A.ny = in.ny;
  A.nz = in.nz;
  A.ng = t.ng;
  A.h = in.h;
  A.d1 = in.prm.d1;
  A.d2 = in.prm.d2;
  A.weights = in.prm.weights;
  A.gcell = t.gcell;
  A.cmap = t.cmap;
  A.alpha_c = t.alpha_c;
  A.nrm = t.nrm;
  A.dn = t.dn;
  A.gamma = t.gamma;
  A.ap1 = t.ap1;
  A.w1 = t.w1;
  A.ap2 = t.ap2;
  A.w2 = t.w2;
  A.n_fallback = counters;
  A.n_fail = counters + 1;
  k_ghost_weights3<<<blocks_for(t.ng, 128), 128, 0, s>>>(A);
  IBPF_TRY3(cudaGetLastError());
  int hc[2] = {0, 0};
  IBPF_TRY3(cudaMemcpyAsync(hc, counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  IBPF_TRY3(cudaStreamSynchronize(s));
  cudaFree(counters);
  t.n_fallback = hc[0];
  *n_fail = hc[1];
  return cudaSuccess;
}

}  // namespace ibpf
