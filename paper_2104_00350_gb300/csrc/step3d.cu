// One time step of the hybrid IB / phase-field method on a 3D staggered grid (Sec. 4.2 and
// Appendix A of arXiv 2104.00350 with the third axis), templated on the field type T.
//
// Layout: cells (k, j, i) at (k ny + j) nx + i; u on x-faces (face i = left face of cell i),
// v on y-faces (face j = front face of cell j), both nz x ny x nx; w on z-faces, (nz+1)
// planes with planes 0 and nz on the walls.  Periodic in x and y; at the z walls C, phi and
// P take mirror planes and the tangential velocities u, v the no-slip ghost planes -u, -v.
// Discrete operators as in 2D: 7-point Laplacian, arithmetic face means, edge viscosities
// from the mean C of the four cells around the edge, divergence-form convection with the
// products of face means at the edges.  The solves work on increments exactly as the 2D
// step does (CH: over the BDF2 predictor B; pressure: over P^ = 2P^n - P^{n-1}).
#include <cmath>
#include <type_traits>
#include <vector>

#include "batch.h"
#include "cell_common.cuh"
#include "ibpf_internal.h"

namespace ibpf {
namespace {

template <typename T>
struct S3 {
  int nx, ny, nz, lnx, lny;
  T inv_h, inv_h2, dt, S, inv_eta2, pe_eta2, inv_dt, eta2;
  T rho_a, rho_b, mu_a, mu_b, rho0, inv_rho0, Re, k_st;
  T inv_pe;   // 1/Pe (explicit Cahn-Hilliard variant)
  double k_wet, cos_th, l_s;
  double a_dyn, inv_ca;    // dynamic angle: dt / (mu_f Cn) (0: static), 1 / Ca
  // fields (level cur is n)
  const T* C;    // C^n
  const T* Co;   // C^{n-1}
  T* C1;         // C^{n+1} (the C^{n-1} slot after the solve)
  T* C1lo;
  const T* Clo;  // low part of C^n (FP32 form)
  const T *U, *V, *W, *Uo, *Vo, *Wo;   // u^n, u^{n-1}
  T *Us, *Vs, *Ws;                     // u** and then u^{n+1} (the n-1 slots)
  T *Hu, *Hv, *Hw;
  const T *P, *Po;
  T *Q, *phi, *rhs, *phat, *dp;
  T *gu, *gv, *gw, *fval;
  double* ci;    // dynamic angle: wall values C_I (state, FP64 in both forms)
  T* gq;         // dynamic angle: scratch C_G, B, (dC/dx_t)_I (3)
  const T *au, *av, *aw;   // face fractions in the field type
  Tables tab;
  double* partial;
  unsigned* ticket;
  double* mass;
  int* status;
  int pred_kz;   // planes per predictor block (a power of two, at most nz)
  const T *w1t, *w2t;   // averaging weights in the field type (FP32: copies of the FP64 ones)
};


template <typename T>
__device__ __forceinline__ void cell_ijk(const S3<T>& a, size_t c, int& i, int& j, int& k) {
  i = (int)(c & (size_t)(a.nx - 1));
  j = (int)((c >> a.lnx) & (size_t)(a.ny - 1));
  k = (int)(c >> (a.lnx + a.lny));
}

// linear indices of the 6 face neighbours of cell c: periodic in x and y, mirror planes in
// z (zp / zm are c itself at the walls)
struct Nbr {
  size_t c, xp, xm, yp, ym, zp, zm;
};
template <typename T>
__device__ __forceinline__ Nbr nbr(const S3<T>& a, size_t c, int i, int j, int k) {
  const size_t nx = (size_t)a.nx, nxy = nx * a.ny;
  Nbr n;
  n.c = c;
  n.xp = i == a.nx - 1 ? c - (nx - 1) : c + 1;
  n.xm = i == 0 ? c + (nx - 1) : c - 1;
  n.yp = j == a.ny - 1 ? c - (nxy - nx) : c + nx;
  n.ym = j == 0 ? c + (nxy - nx) : c - nx;
  n.zp = k == a.nz - 1 ? c : c + nxy;
  n.zm = k == 0 ? c : c - nxy;
  return n;
}

// ------------------------------------------------------------ a3 / a4: ghost fills, phi
template <typename T>
__device__ __forceinline__ T gather7(const T* __restrict__ f, const int* __restrict__ ap,
                                     const T* __restrict__ w, int g) {
  T acc = T(0);
#pragma unroll
  for (int q = 0; q < kNap3; ++q) acc = acc + (T)w[(size_t)g * kNap3 + q] * f[ap[(size_t)g * kNap3 + q]];
  return acc;
}

// Warp-cooperative gathers (the velocity fill, six values per averaging point): each ghost
// gets a group of kGhostLanes = 8 lanes (four ghosts per warp).  Lane q < 7 takes averaging point q of both
// interpolation points: its two stencil entries (the group's entries are contiguous, so the
// table loads coalesce), its field values at the two points and their weighted products; the
// products meet by three xor shuffles, the same tree for every ghost, and every lane of the
// group ends with the sums s1 (IP1) and s2 (IP2).  NV values per point: get(c, v) writes
// them for cell c.  Every lane of the warp calls it (the shuffles need the whole warp);
// lanes of groups past the last ghost contribute zeros.  The one-value fills (C, phi, the
// wall term) stay one thread per ghost: in this form they measured slower (fill_C 125 ->
// 190 us, fill_phi 108 -> 137 us on the 512^3 packing), the velocity fill faster (332 ->
// 293 us).
constexpr int kGhostLanes = 8, kGhostBlock = 256;
template <int NV, typename T, typename Get>
__device__ __forceinline__ void gather_group(const Tables& t, const T* __restrict__ w1t,
                                             const T* __restrict__ w2t, int g, int q, Get get,
                                             T (&s1)[NV], T (&s2)[NV]) {
#pragma unroll
  for (int v = 0; v < NV; ++v) s1[v] = s2[v] = T(0);
  if (g < t.ng && q < kNap3) {
    const size_t e = (size_t)g * kNap3 + q;
    const size_t c1 = (size_t)t.ap1[e], c2 = (size_t)t.ap2[e];
    const T w1 = w1t[e], w2 = w2t[e];
    T v1[NV], v2[NV];
    get(c1, v1);
    get(c2, v2);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      s1[v] = w1 * v1[v];
      s2[v] = w2 * v2[v];
    }
  }
#pragma unroll
  for (int o = 1; o < kGhostLanes; o <<= 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      s1[v] += __shfl_xor_sync(0xffffffffu, s1[v], o);
      s2[v] += __shfl_xor_sync(0xffffffffu, s2[v], o);
    }
  }
}

// static contact angle, the same cut-off rule as the 2D step (see step2d.cu)
template <typename T>
__global__ void k3_fill_C(S3<T> a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const Tables& t = a.tab;
  if (g >= t.ng) return;
  const T cm = T(2) * gather7(a.C1, t.ap1, a.w1t, g) - gather7(a.C1, t.ap2, a.w2t, g);
  const T gam = (T)t.gamma[g], dn = (T)t.dn[g];
  const T kk = (T)a.k_wet / (gam * dn);
  const T qa = T(-0.75) * (T)a.cos_th;
  const T qc = kk * cm + T(0.75) * (T)a.cos_th;
  T disc = kk * kk - T(4) * qa * qc;
  disc = disc > T(0) ? disc : T(0);
  const T sq = sqrt(disc);
  T ci = T(2) * qc / (kk + sq);
  if (!(fabs(ci) <= T(1)) && qa != T(0)) {
    ci = (kk + sq) / (T(2) * qa);
    ci = ci > T(1) ? T(1) : (ci < T(-1) ? T(-1) : ci);
  }
  if (fabs(cm) >= T(1)) ci = cm;
  a.C1[t.gcell[g]] = ((gam + T(1)) * ci - cm) / gam;
  if (a.C1lo) a.C1lo[t.gcell[g]] = T(0);
}

// dynamic angle (mu_f > 0): Eq. WallBCS_recast for the per-ghost state C_I, as the 2D step
// (step2d.cu, fill_C_dynamic) with the vector forms v_t (dC/dx_t) = V_t . grad C and
// (dC/dx_t)_I = grad C - (grad C . n) n; pass 0 computes into scratch, pass 1 writes the ghosts
template <typename T>
__device__ __forceinline__ T cen3(const S3<T>& a, const T* __restrict__ f, size_t c, int axis) {
  if (axis == 0) {
    const int i = (int)(c & (size_t)(a.nx - 1));
    return T(0.5) * (f[c] + f[c - i + ((i + 1) & (a.nx - 1))]);
  }
  if (axis == 1) {
    const int j = (int)((c >> a.lnx) & (size_t)(a.ny - 1));
    const size_t row0 = c - ((size_t)j << a.lnx);
    return T(0.5) * (f[c] + f[row0 + ((size_t)((j + 1) & (a.ny - 1)) << a.lnx)]);
  }
  return T(0.5) * (f[c] + f[c + ((size_t)a.nx << a.lny)]);
}

template <typename T>
__device__ __forceinline__ void cgrad3(const S3<T>& a, const T* __restrict__ C, size_t c, T* g) {
  int i, j, k;
  cell_ijk(a, c, i, j, k);
  const Nbr n = nbr(a, c, i, j, k);
  const T hh = T(0.5) * a.inv_h;
  g[0] = (C[n.xp] - C[n.xm]) * hh;
  g[1] = (C[n.yp] - C[n.ym]) * hh;
  g[2] = (C[n.zp] - C[n.zm]) * hh;
}

template <typename T>
__global__ void k3_fill_Cd(S3<T> a, int pass) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const Tables& t = a.tab;
  const int ng = t.ng;
  if (g >= ng) return;
  if (pass == 1) {
    a.C1[t.gcell[g]] = a.gq[g];
    if (a.C1lo) a.C1lo[t.gcell[g]] = T(0);
    return;
  }
  T m1 = T(0), m2 = T(0), n1c = T(0), n2c = T(0);
  T U1[3] = {T(0), T(0), T(0)}, U2[3] = {T(0), T(0), T(0)};
  T G1[3] = {T(0), T(0), T(0)}, G2[3] = {T(0), T(0), T(0)};
  const T* uf[3] = {a.U, a.V, a.W};
#pragma unroll
  for (int q = 0; q < kNap3; ++q) {
    const size_t c1 = t.ap1[(size_t)g * kNap3 + q], c2 = t.ap2[(size_t)g * kNap3 + q];
    const T w1 = a.w1t[(size_t)g * kNap3 + q], w2 = a.w2t[(size_t)g * kNap3 + q];
    m1 = m1 + w1 * a.C1[c1];
    m2 = m2 + w2 * a.C1[c2];
    n1c = n1c + w1 * a.C[c1];
    n2c = n2c + w2 * a.C[c2];
    T g1[3], g2[3];
    cgrad3(a, (const T*)a.C1, c1, g1);
    cgrad3(a, (const T*)a.C1, c2, g2);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      U1[d] = U1[d] + w1 * cen3(a, uf[d], c1, d);
      U2[d] = U2[d] + w2 * cen3(a, uf[d], c2, d);
      G1[d] = G1[d] + w1 * g1[d];
      G2[d] = G2[d] + w2 * g2[d];
    }
  }
  const size_t cg = (size_t)t.gcell[g];
  // the wall value is state: held and updated in FP64 in both forms (see step2d.cu)
  const double gam = t.gamma[g], dn = t.dn[g];
  const double gp1 = gam + 1.0;
  const double cm = 2.0 * (double)m1 - (double)m2;
  double ci_n = a.ci[g];
  if (!isfinite(ci_n)) ci_n = (gam * (double)a.C[cg] + (2.0 * (double)n1c - (double)n2c)) / gp1;
  T gG[3];
  cgrad3(a, (const T*)a.C1, cg, gG);
  const T nn[3] = {(T)t.nrm[3 * (size_t)g], (T)t.nrm[3 * (size_t)g + 1], (T)t.nrm[3 * (size_t)g + 2]};
  const T tg = (T)gam, tp1 = (T)gp1;
  T UI[3], GI[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    UI[d] = (tg * cen3(a, uf[d], cg, d) + (T(2) * U1[d] - U2[d])) / tp1;
    GI[d] = (tg * gG[d] + (T(2) * G1[d] - G2[d])) / tp1;
  }
  const T un = (UI[0] * nn[0] + UI[1] * nn[1]) + UI[2] * nn[2];
  const T gn = (GI[0] * nn[0] + GI[1] * nn[1]) + GI[2] * nn[2];
  T gt[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) gt[d] = GI[d] - gn * nn[d];
  T advT;
  {
    const T vt0 = UI[0] - un * nn[0], vt1 = UI[1] - un * nn[1], vt2 = UI[2] - un * nn[2];
    advT = (vt0 * GI[0] + vt1 * GI[1]) + vt2 * GI[2];
  }
  const double adv = (double)advT;
  const double ct = a.cos_th, aa = a.a_dyn;
  const double k = a.k_wet / (gam * dn);
  const double R = (ci_n - (double)a.dt * adv) + aa * k * cm;
  const double qb = 1.0 + aa * k;
  const double lin = R / qb;
  const double qa = 0.75 * aa * ct;
  const double qc = R + 0.75 * aa * ct;
  double disc = qb * qb + 4.0 * qa * qc;
  disc = disc > 0.0 ? disc : 0.0;
  const double sq = sqrt(disc);
  double cI = 2.0 * qc / (qb + sq);
  if (!(fabs(cI) <= 1.0) && qa != 0.0) {
    cI = -(qb + sq) / (2.0 * qa);
    cI = cI > 1.0 ? 1.0 : (cI < -1.0 ? -1.0 : cI);
  }
  if (fabs(lin) >= 1.0) cI = lin;
  const double gpr = fabs(cI) < 1.0 ? 0.75 * (1.0 - cI * cI) : 0.0;
  a.ci[g] = cI;
  a.gq[g] = (T)((gp1 * cI - cm) / gam);
  a.gq[ng + g] = (T)(k * (cm - cI) + ct * gpr);
  a.gq[2 * ng + g] = gt[0];
  a.gq[3 * ng + g] = gt[1];
  a.gq[4 * ng + g] = gt[2];
}

// a1, wall term: the wall's no-flux condition d(phi)/dn = 0 (Eq. AllBCs) on the chemical
// potential phi~ = psi'(C~) - Cn^2 lap(C~) of C~ = 2C^n - C^{n-1} (written by ch_h into the
// rhs scratch), imposed by the ghost fill phi~_G = phi~_M of Sec. 4.2.2: h_G += (phi~_M -
// phi~_G)/Cn^2 (as the 2D step; only ghost entries of h change, phi~ is only read)
template <typename T>
__global__ void k3_ch_wall(S3<T> a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const Tables& t = a.tab;
  if (g >= t.ng) return;
  const T pm = T(2) * gather7((const T*)a.rhs, t.ap1, a.w1t, g) - gather7((const T*)a.rhs, t.ap2, a.w2t, g);
  const size_t c = (size_t)t.gcell[g];
  a.phi[c] = a.phi[c] + (pm - a.rhs[c]) * a.inv_eta2;
}

// zero normal gradient of phi at the wall: phi_G = phi_M
template <typename T>
__global__ void k3_fill_phi(S3<T> a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const Tables& t = a.tab;
  if (g >= t.ng) return;
  a.phi[t.gcell[g]] = T(2) * gather7(a.phi, t.ap1, a.w1t, g) - gather7(a.phi, t.ap2, a.w2t, g);
}

// --------------------------------------- four-cells-per-thread kernels (FP32 form)
// Thread t owns the x-run of cells 4t .. 4t+3 (one 16-byte word per field and row); the
// y and z neighbours are the words one row or one plane away, the x neighbours of the run
// come from the adjacent lanes by shuffles (or a load at a row end or a warp end).  The
// arithmetic of each cell is that of the z-marching kernels below (the FP64 form), term for
// term.  For the FP32 form, which is memory-latency bound, these measured faster on GB300
// than one thread per cell (by 1.5-2.2x) and than the z-marching windows.
constexpr int kTQ = 128;   // threads per block: 512 cells, the smallest grid has 512 cells

// the run of a thread: first cell q (i0 = q mod nx), its row / plane offsets for the y and z
// neighbours (periodic in y; the run itself at the z walls), and the linear indices of the
// left neighbour of cell 0 and the right neighbour of cell 3 (periodic in x)
struct Run {
  size_t q, ym, yp, zm, zp, xl, xr;
  int i0, j, k, lane;
};
__device__ __forceinline__ Run run4(const S3<float>& a) {
  Run r;
  r.q = ((size_t)blockIdx.x * kTQ + threadIdx.x) * 4;
  cell_ijk(a, r.q, r.i0, r.j, r.k);
  const size_t nx = (size_t)a.nx, nxy = nx * a.ny;
  r.lane = threadIdx.x & 31;
  r.xl = r.i0 == 0 ? r.q + (nx - 1) : r.q - 1;
  r.xr = r.i0 + 4 == a.nx ? r.q + 4 - nx : r.q + 4;
  r.yp = r.j == a.ny - 1 ? r.q - (nxy - nx) : r.q + nx;
  r.ym = r.j == 0 ? r.q + (nxy - nx) : r.q - nx;
  r.zp = r.k == a.nz - 1 ? r.q : r.q + nxy;
  r.zm = r.k == 0 ? r.q : r.q - nxy;
  return r;
}

template <typename G>
__device__ __forceinline__ X2 xnb(const V4& v, const Run& d, int nx, G g) {
  return xnb<32>(v, d.lane, d.i0 == 0, d.i0 + 4 == nx, d.xl, d.xr, g);
}

// 7-point Laplacian of cell e of the run (xm + xp first, as lap7)
__device__ __forceinline__ float lap7q(const S3<float>& a, const V4& c, const X2& x, const V4& yp,
                                       const V4& ym, const V4& zp, const V4& zm, int e) {
  return ((((right(c, x, e) + left(c, x, e)) + (yp.e[e] + ym.e[e])) + (zp.e[e] + zm.e[e])) -
          6.0f * c.e[e]) * a.inv_h2;
}

// a1: h = (psi'(C~) - S (C~ - B))/Cn^2 - lap(B), B = C^n + (C^n - C^{n-1})/3, C~ - B = 2 d/3
__global__ void __launch_bounds__(kTQ) k3_ch_h_q(S3<float> a) {
  const Run d = run4(a);
  const float third = float(1.0 / 3.0);
  auto Bq = [&](size_t q) { return a.C[q] + (a.C[q] - a.Co[q]) * third; };
  auto Bv = [&](const V4& c, const V4& o) {
    return map4([&](int e) { return c.e[e] + (c.e[e] - o.e[e]) * third; });
  };
  // C and C_old at the run and its y / z neighbours, loaded once for h and (with ghosts) phi~
  const V4 c = ld4(a.C, d.q), o = ld4(a.Co, d.q);
  const V4 cyp = ld4(a.C, d.yp), oyp = ld4(a.Co, d.yp), cym = ld4(a.C, d.ym), oym = ld4(a.Co, d.ym);
  const V4 czp = ld4(a.C, d.zp), ozp = ld4(a.Co, d.zp), czm = ld4(a.C, d.zm), ozm = ld4(a.Co, d.zm);
  const V4 b = Bv(c, o);
  const V4 byp = Bv(cyp, oyp), bym = Bv(cym, oym), bzp = Bv(czp, ozp), bzm = Bv(czm, ozm);
  const X2 bx = xnb(b, d, a.nx, Bq);
  st4(a.phi, d.q, map4([&](int e) {
        const float lapb = lap7q(a, b, bx, byp, bym, bzp, bzm, e);
        const float dd = c.e[e] - o.e[e];
        const float ct = c.e[e] + dd;
        return ((ct * ct * ct - ct) - a.S * (2.0f * third * dd)) * a.inv_eta2 - lapb;
      }));
  if (a.tab.ng > 0) {
    // phi~ = psi'(C~) - Cn^2 lap(C~) for the wall term (k3_ch_wall), into the rhs scratch
    auto Tv = [&](const V4& x, const V4& y) {
      return map4([&](int e) { return 2.0f * x.e[e] - y.e[e]; });
    };
    const V4 ct = Tv(c, o);
    const V4 typ = Tv(cyp, oyp), tym = Tv(cym, oym), tzp = Tv(czp, ozp), tzm = Tv(czm, ozm);
    const X2 tx = xnb(ct, d, a.nx, [&](size_t q) { return 2.0f * a.C[q] - a.Co[q]; });
    st4(a.rhs, d.q, map4([&](int e) {
          const float x = ct.e[e];
          return (x * x * x - x) - a.eta2 * lap7q(a, ct, tx, typ, tym, tzp, tzm, e);
        }));
  }
}

// a1: R = lap(h) - (Pe/Cn^2) div(u~ C~), u~ = 2u^n - u^{n-1}, C~ = 2C^n - C^{n-1}; no flux
// through the z walls
__global__ void __launch_bounds__(kTQ) k3_ch_rhs_q(S3<float> a) {
  const Run d = run4(a);
  const size_t nxy = (size_t)a.nx * a.ny;
  auto two = [&](const float* f, const float* fo, size_t q) {
    const V4 x = ld4(f, q), y = ld4(fo, q);
    return map4([&](int e) { return 2.0f * x.e[e] - y.e[e]; });
  };
  auto ctq = [&](size_t q) { return 2.0f * a.C[q] - a.Co[q]; };
  auto utq = [&](size_t q) { return 2.0f * a.U[q] - a.Uo[q]; };
  const V4 c0 = two(a.C, a.Co, d.q), cyp = two(a.C, a.Co, d.yp), cym = two(a.C, a.Co, d.ym);
  const V4 czp = two(a.C, a.Co, d.zp), czm = two(a.C, a.Co, d.zm);
  const V4 ut = two(a.U, a.Uo, d.q), vt = two(a.V, a.Vo, d.q), vtn = two(a.V, a.Vo, d.yp);
  const V4 wt = two(a.W, a.Wo, d.q), wtt = two(a.W, a.Wo, d.q + nxy);
  const V4 h = ld4(a.phi, d.q), hyp = ld4(a.phi, d.yp), hym = ld4(a.phi, d.ym);
  const V4 hzp = ld4(a.phi, d.zp), hzm = ld4(a.phi, d.zm);
  const X2 cx = xnb(c0, d, a.nx, ctq), ux = xnb(ut, d, a.nx, utq);
  const X2 hx = xnb(h, d, a.nx, [&](size_t q) { return a.phi[q]; });
  st4(a.Q, d.q, map4([&](int e) {
        const float cc = c0.e[e];
        const float fx_w = ut.e[e] * (0.5f * (left(c0, cx, e) + cc));
        const float fx_e = right(ut, ux, e) * (0.5f * (cc + right(c0, cx, e)));
        const float fy_s = vt.e[e] * (0.5f * (cym.e[e] + cc));
        const float fy_n = vtn.e[e] * (0.5f * (cc + cyp.e[e]));
        const float fz_b = d.k > 0 ? wt.e[e] * (0.5f * (czm.e[e] + cc)) : 0.0f;
        const float fz_t = d.k < a.nz - 1 ? wtt.e[e] * (0.5f * (cc + czp.e[e])) : 0.0f;
        const float div = ((fx_e - fx_w) * a.inv_h + (fy_n - fy_s) * a.inv_h) + (fz_t - fz_b) * a.inv_h;
        return lap7q(a, h, hx, hyp, hym, hzp, hzm, e) - a.pe_eta2 * div;
      }));
}

// a4: phi = psi'(C) - Cn^2 lap C on every cell
__global__ void __launch_bounds__(kTQ) k3_chem_pot_q(S3<float> a) {
  const Run d = run4(a);
  const V4 c = ld4(a.C1, d.q);
  const V4 cyp = ld4(a.C1, d.yp), cym = ld4(a.C1, d.ym), czp = ld4(a.C1, d.zp), czm = ld4(a.C1, d.zm);
  const X2 cx = xnb(c, d, a.nx, [&](size_t q) { return a.C1[q]; });
  st4(a.phi, d.q, map4([&](int e) {
        const float c0 = c.e[e];
        return (c0 * c0 * c0 - c0) - a.eta2 * lap7q(a, c, cx, cyp, cym, czp, czm, e);
      }));
}

// a7: lap dP = (rho0/dt) div u** - div[(rho0/rho_f) grad P^], dP = P^{n+1} - P^; stores P^
__global__ void __launch_bounds__(kTQ, 6) k3_poisson_rhs_q(S3<float> a) {
  const Run d = run4(a);
  const size_t nxy = (size_t)a.nx * a.ny;
  auto rho = [&](float cc) { return a.rho_a + a.rho_b * clamp1(cc); };
  auto ph4 = [&](size_t q) {
    const V4 p = ld4(a.P, q), po = ld4(a.Po, q);
    return map4([&](int e) { return 2.0f * p.e[e] - po.e[e]; });
  };
  const float* C = a.C1;
  const V4 p0 = ph4(d.q), pyp = ph4(d.yp), pym = ph4(d.ym), pzp = ph4(d.zp), pzm = ph4(d.zm);
  const V4 c0 = ld4(C, d.q), cyp = ld4(C, d.yp), cym = ld4(C, d.ym), czp = ld4(C, d.zp), czm = ld4(C, d.zm);
  const V4 us = ld4(a.Us, d.q), vs = ld4(a.Vs, d.q), vsn = ld4(a.Vs, d.yp);
  const V4 ws = ld4(a.Ws, d.q), wst = ld4(a.Ws, d.q + nxy);
  const X2 px = xnb(p0, d, a.nx, [&](size_t q) { return 2.0f * a.P[q] - a.Po[q]; });
  const X2 cx = xnb(c0, d, a.nx, [&](size_t q) { return C[q]; });
  const X2 ux = xnb(us, d, a.nx, [&](size_t q) { return a.Us[q]; });
  V4 rhs, phat;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float pc = p0.e[e], cc = c0.e[e];
    const float gx_w = qdiv(a.rho0, rho(0.5f * (left(c0, cx, e) + cc))) * ((pc - left(p0, px, e)) * a.inv_h);
    const float gx_e = qdiv(a.rho0, rho(0.5f * (cc + right(c0, cx, e)))) * ((right(p0, px, e) - pc) * a.inv_h);
    const float gy_s = qdiv(a.rho0, rho(0.5f * (cym.e[e] + cc))) * ((pc - pym.e[e]) * a.inv_h);
    const float gy_n = qdiv(a.rho0, rho(0.5f * (cc + cyp.e[e]))) * ((pyp.e[e] - pc) * a.inv_h);
    float gz_b = 0.0f, gz_t = 0.0f;
    if (d.k > 0) gz_b = qdiv(a.rho0, rho(0.5f * (czm.e[e] + cc))) * ((pc - pzm.e[e]) * a.inv_h);
    if (d.k < a.nz - 1) gz_t = qdiv(a.rho0, rho(0.5f * (cc + czp.e[e]))) * ((pzp.e[e] - pc) * a.inv_h);
    const float div_g = ((gx_e - gx_w) * a.inv_h + (gy_n - gy_s) * a.inv_h) + (gz_t - gz_b) * a.inv_h;
    const float div_u = ((right(us, ux, e) - us.e[e]) * a.inv_h + (vsn.e[e] - vs.e[e]) * a.inv_h) +
                        (wst.e[e] - ws.e[e]) * a.inv_h;
    rhs.e[e] = (a.rho0 * a.inv_dt) * div_u - div_g;
    phat.e[e] = pc;
  }
  st4(a.rhs, d.q, rhs);
  st4(a.phat, d.q, phat);
}

// a8: u^{n+1} = u** - dt [ (1/rho_f) grad P^ + (1/rho0) grad dP ] on every face (z-faces
// 1..nz-1); non-finite check; the tile's compensated sum of C for the FP64 mass
__global__ void __launch_bounds__(kTQ, 10) k3_correct_q(S3<float> a) {
  const Run d = run4(a);
  auto rho = [&](float cc) { return a.rho_a + a.rho_b * clamp1(cc); };
  const float* C = a.C1;
  const V4 c0 = ld4(C, d.q), cym = ld4(C, d.ym), czm = ld4(C, d.zm);
  const V4 ph = ld4(a.phat, d.q), phym = ld4(a.phat, d.ym), phzm = ld4(a.phat, d.zm);
  const V4 dp = ld4(a.dp, d.q), dpym = ld4(a.dp, d.ym), dpzm = ld4(a.dp, d.zm);
  const V4 us = ld4(a.Us, d.q), vs = ld4(a.Vs, d.q);
  const X2 cx = xnb(c0, d, a.nx, [&](size_t q) { return C[q]; });
  const X2 phx = xnb(ph, d, a.nx, [&](size_t q) { return a.phat[q]; });
  const X2 dpx = xnb(dp, d, a.nx, [&](size_t q) { return a.dp[q]; });
  const bool top = d.k >= 1;
  V4 ws = {{0.0f, 0.0f, 0.0f, 0.0f}};
  if (top) ws = ld4(a.Ws, d.q);
  int bad = 0;
  auto corr = [&](float vel, float cn, float cc, float phn, float phc, float dpn, float dpc) {
    const float rho_f = rho(0.5f * (cn + cc));
    const float vn = vel - a.dt * (qdiv((phc - phn) * a.inv_h, rho_f) + a.inv_rho0 * ((dpc - dpn) * a.inv_h));
    bad |= !isfinite(vn);
    return vn;
  };
  V4 un, vn, wn;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float cc = c0.e[e], pc = ph.e[e], dc = dp.e[e];
    un.e[e] = corr(us.e[e], left(c0, cx, e), cc, left(ph, phx, e), pc, left(dp, dpx, e), dc);
    vn.e[e] = corr(vs.e[e], cym.e[e], cc, phym.e[e], pc, dpym.e[e], dc);
    wn.e[e] = top ? corr(ws.e[e], czm.e[e], cc, phzm.e[e], pc, dpzm.e[e], dc) : 0.0f;
    bad |= !isfinite(cc);
  }
  st4(a.Us, d.q, un);
  st4(a.Vs, d.q, vn);
  if (top) st4(a.Ws, d.q, wn);
  if (bad) atomicOr(a.status, 1);
  const V4 lo = a.C1lo ? ld4(a.C1lo, d.q) : V4{{0.0f, 0.0f, 0.0f, 0.0f}};
  float hi = c0.e[0], lsum = lo.e[0];
#pragma unroll
  for (int e = 1; e < 4; ++e) pair_add(hi, lsum, c0.e[e], lo.e[e]);
  // one FP64 partial per warp (no block barrier); k3_mass_groups / k3_mass_total add them
  warp_pair_sum(hi, lsum);
  if ((threadIdx.x & 31) == 0)
    a.partial[(size_t)blockIdx.x * (kTQ / 32) + (threadIdx.x >> 5)] = (double)hi + (double)lsum;
}

// The FP64 mass of the FP32 3D step from the correction kernel's warp partials: kMassSpan
// partials per block in a fixed tree, then the block sums by one block, in a fixed order.
constexpr int kMassSpan = 1024, kMassThreads = 256;
__global__ void __launch_bounds__(kMassThreads) k3_mass_groups(const double* __restrict__ partial,
                                                               int n, double* __restrict__ gsum) {
  __shared__ double wd[kMassThreads / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < kMassSpan; i += kMassThreads) {
    const size_t e = (size_t)blockIdx.x * kMassSpan + i;
    if (e < (size_t)n) v += partial[e];
  }
  v = block_sum<kMassThreads>(v, wd);
  if (threadIdx.x == 0) gsum[blockIdx.x] = v;
}
__global__ void __launch_bounds__(kMassThreads) k3_mass_total(const double* __restrict__ gsum, int n,
                                                              double* __restrict__ mass) {
  __shared__ double wd[kMassThreads / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += kMassThreads) v += gsum[i];
  v = block_sum<kMassThreads>(v, wd);
  if (threadIdx.x == 0) *mass = v;
}

// ------------------------------------- a1 + a2, explicit variant (Eq. ExpCH), 3D
// The 2D variant with the third axis: C^{n+1} = C^n + dt (3/2 F^n - 1/2 F^{n-1}),
// F = -div(u C_f) + (1/Pe) lap(phi), F^{n-1} from the level n-1 fields, phi at both levels
// with their ghost fills.  k3x_phi2 writes phi^n -> phi, phi^{n-1} -> rhs and
// A^{n-1} = -div(u^{n-1} C^{n-1}_f) -> Q; k3x_fill2 fills the ghosts of phi and rhs;
// k3x_update writes C^{n+1} into the C^{n-1} slot (compensated in FP32), reading C^{n-1}
// only through Q and rhs.  FP64: one thread per cell; FP32: runs of four cells.
constexpr int kTX = 256;

template <typename T>
__device__ __forceinline__ T lap7x(const S3<T>& a, const T* __restrict__ f, const Nbr& n) {
  return ((((f[n.xp] + f[n.xm]) + (f[n.yp] + f[n.ym])) + (f[n.zp] + f[n.zm])) - T(6) * f[n.c]) *
         a.inv_h2;
}

template <typename T>
__device__ __forceinline__ T flux_div3(const S3<T>& a, const T* __restrict__ C, const T* __restrict__ u,
                                       const T* __restrict__ v, const T* __restrict__ w,
                                       const Nbr& n, int k) {
  const size_t c = n.c, nxy = (size_t)a.nx * a.ny;
  const T c0 = C[c];
  const T fx_w = u[c] * (T(0.5) * (C[n.xm] + c0));
  const T fx_e = u[n.xp] * (T(0.5) * (c0 + C[n.xp]));
  const T fy_s = v[c] * (T(0.5) * (C[n.ym] + c0));
  const T fy_n = v[n.yp] * (T(0.5) * (c0 + C[n.yp]));
  const T fz_b = k > 0 ? w[c] * (T(0.5) * (C[c - nxy] + c0)) : T(0);
  const T fz_t = k < a.nz - 1 ? w[c + nxy] * (T(0.5) * (c0 + C[c + nxy])) : T(0);
  return ((fx_e - fx_w) * a.inv_h + (fy_n - fy_s) * a.inv_h) + (fz_t - fz_b) * a.inv_h;
}

template <typename T>
__global__ void __launch_bounds__(kTX) k3x_phi2(S3<T> a) {
  const size_t c = (size_t)blockIdx.x * kTX + threadIdx.x;
  int i, j, k;
  cell_ijk(a, c, i, j, k);
  const Nbr n = nbr(a, c, i, j, k);
  const T cn = a.C[c], co = a.Co[c];
  const T pn = (cn * cn * cn - cn) - a.eta2 * lap7x(a, a.C, n);
  const T po = (co * co * co - co) - a.eta2 * lap7x(a, a.Co, n);
  const T ao = -flux_div3(a, a.Co, a.Uo, a.Vo, a.Wo, n, k);
  a.phi[c] = pn;
  a.rhs[c] = po;
  a.Q[c] = ao;
}

template <typename T>
__global__ void k3x_fill2(S3<T> a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const Tables& t = a.tab;
  if (g >= t.ng) return;
  a.phi[t.gcell[g]] = T(2) * gather7(a.phi, t.ap1, a.w1t, g) - gather7(a.phi, t.ap2, a.w2t, g);
  a.rhs[t.gcell[g]] = T(2) * gather7(a.rhs, t.ap1, a.w1t, g) - gather7(a.rhs, t.ap2, a.w2t, g);
}

template <typename T>
__global__ void __launch_bounds__(kTX) k3x_update(S3<T> a) {
  const size_t c = (size_t)blockIdx.x * kTX + threadIdx.x;
  int i, j, k;
  cell_ijk(a, c, i, j, k);
  const Nbr n = nbr(a, c, i, j, k);
  const T Fn = -flux_div3(a, a.C, a.U, a.V, a.W, n, k) + lap7x(a, a.phi, n) * a.inv_pe;
  const T Fo = a.Q[c] + lap7x(a, a.rhs, n) * a.inv_pe;
  T hi = a.C[c], lo = a.Clo ? a.Clo[c] : T(0);
  pair_add(hi, lo, a.dt * (T(1.5) * Fn - T(0.5) * Fo), T(0));
  a.C1[c] = hi;
  if (a.C1lo) a.C1lo[c] = lo;
}

// FP32: runs of four cells
__device__ __forceinline__ float flux_div3q(const S3<float>& a, const Run& d, const V4& c, const X2& cx,
                                            const V4& cyp, const V4& cym, const V4& czp, const V4& czm,
                                            const V4& u, const X2& ux, const V4& v, const V4& vn,
                                            const V4& w, const V4& wt, int e) {
  const float c0 = c.e[e];
  const float fx_w = u.e[e] * (0.5f * (left(c, cx, e) + c0));
  const float fx_e = right(u, ux, e) * (0.5f * (c0 + right(c, cx, e)));
  const float fy_s = v.e[e] * (0.5f * (cym.e[e] + c0));
  const float fy_n = vn.e[e] * (0.5f * (c0 + cyp.e[e]));
  const float fz_b = d.k > 0 ? w.e[e] * (0.5f * (czm.e[e] + c0)) : 0.0f;
  const float fz_t = d.k < a.nz - 1 ? wt.e[e] * (0.5f * (c0 + czp.e[e])) : 0.0f;
  return ((fx_e - fx_w) * a.inv_h + (fy_n - fy_s) * a.inv_h) + (fz_t - fz_b) * a.inv_h;
}

__global__ void __launch_bounds__(kTQ) k3x_phi2_q(S3<float> a) {
  const Run d = run4(a);
  const size_t nxy = (size_t)a.nx * a.ny;
  const V4 c = ld4(a.C, d.q), cyp = ld4(a.C, d.yp), cym = ld4(a.C, d.ym), czp = ld4(a.C, d.zp), czm = ld4(a.C, d.zm);
  const V4 o = ld4(a.Co, d.q), oyp = ld4(a.Co, d.yp), oym = ld4(a.Co, d.ym), ozp = ld4(a.Co, d.zp), ozm = ld4(a.Co, d.zm);
  const V4 u = ld4(a.Uo, d.q), v = ld4(a.Vo, d.q), vn = ld4(a.Vo, d.yp);
  const V4 w = ld4(a.Wo, d.q), wt = ld4(a.Wo, d.q + nxy);
  const X2 cx = xnb(c, d, a.nx, [&](size_t q) { return a.C[q]; });
  const X2 ox = xnb(o, d, a.nx, [&](size_t q) { return a.Co[q]; });
  const X2 ux = xnb(u, d, a.nx, [&](size_t q) { return a.Uo[q]; });
  const V4 pn = map4([&](int e) {
    const float c0 = c.e[e];
    return (c0 * c0 * c0 - c0) - a.eta2 * lap7q(a, c, cx, cyp, cym, czp, czm, e);
  });
  const V4 po = map4([&](int e) {
    const float c0 = o.e[e];
    return (c0 * c0 * c0 - c0) - a.eta2 * lap7q(a, o, ox, oyp, oym, ozp, ozm, e);
  });
  const V4 ao = map4([&](int e) { return -flux_div3q(a, d, o, ox, oyp, oym, ozp, ozm, u, ux, v, vn, w, wt, e); });
  st4(a.phi, d.q, pn);
  st4(a.rhs, d.q, po);
  st4(a.Q, d.q, ao);
}

__global__ void __launch_bounds__(kTQ) k3x_update_q(S3<float> a) {
  const Run d = run4(a);
  const size_t nxy = (size_t)a.nx * a.ny;
  const V4 c = ld4(a.C, d.q), cyp = ld4(a.C, d.yp), cym = ld4(a.C, d.ym), czp = ld4(a.C, d.zp), czm = ld4(a.C, d.zm);
  const V4 u = ld4(a.U, d.q), v = ld4(a.V, d.q), vn = ld4(a.V, d.yp);
  const V4 w = ld4(a.W, d.q), wt = ld4(a.W, d.q + nxy);
  const V4 f = ld4(a.phi, d.q), fyp = ld4(a.phi, d.yp), fym = ld4(a.phi, d.ym), fzp = ld4(a.phi, d.zp), fzm = ld4(a.phi, d.zm);
  const V4 g = ld4(a.rhs, d.q), gyp = ld4(a.rhs, d.yp), gym = ld4(a.rhs, d.ym), gzp = ld4(a.rhs, d.zp), gzm = ld4(a.rhs, d.zm);
  const V4 ao = ld4(a.Q, d.q);
  const V4 lo = a.Clo ? ld4(a.Clo, d.q) : V4{{0.0f, 0.0f, 0.0f, 0.0f}};
  const X2 cx = xnb(c, d, a.nx, [&](size_t q) { return a.C[q]; });
  const X2 ux = xnb(u, d, a.nx, [&](size_t q) { return a.U[q]; });
  const X2 fx = xnb(f, d, a.nx, [&](size_t q) { return a.phi[q]; });
  const X2 gx = xnb(g, d, a.nx, [&](size_t q) { return a.rhs[q]; });
  V4 hi, nlo;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float Fn = -flux_div3q(a, d, c, cx, cyp, cym, czp, czm, u, ux, v, vn, w, wt, e) +
                     lap7q(a, f, fx, fyp, fym, fzp, fzm, e) * a.inv_pe;
    const float Fo = ao.e[e] + lap7q(a, g, gx, gyp, gym, gzp, gzm, e) * a.inv_pe;
    float h = c.e[e], l = lo.e[e];
    pair_add(h, l, a.dt * (1.5f * Fn - 0.5f * Fo), 0.0f);
    hi.e[e] = h;
    nlo.e[e] = l;
  }
  st4(a.C1, d.q, hi);
  if (a.C1lo) st4(a.C1lo, d.q, nlo);
}

// ------------------------------------------------- a5: AB2 predictor + penalisation (3D)
// H = -div(u u) + div(mu (grad u + grad u^T)) / (Re rho_f)
// u* = u^n + dt (3/2 H^n - 1/2 H^{n-1} + (kappa/(Re Ca Cn)) phi_f dC/dn_f / rho_f), u** = alpha_f u*
// Block: a 32 x 8 column of cells marching up kPz planes in z.  Planes k-1, k, k+1 of C, u,
// v, w (and k-1, k of phi) sit in shared memory with a one-cell halo in x and y (periodic
// wrap; mirror planes of C, no-slip ghost planes -u, -v beyond the z walls), so every value
// is read from global memory once per block.  Thread (i, j) updates x-face (i, j, k),
// y-face (i, j, k) and, for k >= 1, z-face (i, j, k) of each plane.
// Edges: xy-edge (i-1/2, j-1/2, k), xz-edge (i-1/2, j, k-1/2), yz-edge (i, j-1/2, k-1/2).
constexpr int kPx = 32, kPy = 8, kPz = 16;
constexpr int kPhx = kPx + 2, kPhy = kPy + 2;

// FP32 form of the predictor: the same blocks, arithmetic and stores, with the staging made
// asynchronous.  Planes go through a ring of four shared-memory slots filled by cp.async
// (no registers held in flight): while plane k is computed the copies of plane k+2 are
// outstanding.  The ghost planes beyond the z walls are staged unsigned (C, u, v of the
// mirrored plane, w and phi zero-filled) and the no-slip sign of u and v is applied on
// reading.
constexpr int kPr = 4;   // ring slots: planes k-1, k, k+1 in use, k+2 arriving

template <typename T>
__device__ __forceinline__ void cp_async_el(T* smem, const T* g, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(g), "n"((int)sizeof(T)),
               "r"(valid ? (int)sizeof(T) : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T>
__global__ void __launch_bounds__(kPx * kPy, 4) k3_predict_a(S3<T> a) {
  __shared__ T sC[kPr][kPhy][kPhx], sU[kPr][kPhy][kPhx], sV[kPr][kPhy][kPhx], sW[kPr][kPhy][kPhx];
  __shared__ T sF[kPr][kPhy][kPhx];
  constexpr int kSlots = kPhx * kPhy, kThreads = kPx * kPy;
  constexpr int NS = (kSlots + kThreads - 1) / kThreads;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPx + tx;
  const int i0 = blockIdx.x * kPx, j0 = blockIdx.y * kPy;
  const int kz = a.pred_kz;
  const int k0 = blockIdx.z * kz;
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < a.nx && j < a.ny;
  const size_t nxy = (size_t)a.nx * a.ny;
  // this thread's staged slots and the in-plane offsets of their columns (periodic wrap)
  unsigned off[NS];
  int sidx[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const int idx = tid + q * kThreads;
    sidx[q] = idx < kSlots ? idx : -1;
    const int r = idx / kPhx, cc = idx % kPhx;
    const int gi = (i0 - 1 + cc + a.nx) & (a.nx - 1), gj = (j0 - 1 + r + a.ny) & (a.ny - 1);
    off[q] = (unsigned)gj * (unsigned)a.nx + (unsigned)gi;
  }
  auto issue = [&](int kk) {   // plane kk (-1 .. nz+1) into slot kk mod 4
    const int sl = (kk + kPr) & (kPr - 1);
    const int km = kk < 0 ? 0 : (kk >= a.nz ? a.nz - 1 : kk);
    const bool win = kk >= 0 && kk <= a.nz, fin = kk >= 0 && kk < a.nz;
    const size_t base = (size_t)km * nxy, wbase = (size_t)(win ? kk : 0) * nxy;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      if (sidx[q] < 0) continue;
      const int e = sl * kSlots + sidx[q];
      cp_async_el(&sC[0][0][0] + e, a.C1 + base + off[q], true);
      cp_async_el(&sU[0][0][0] + e, a.U + base + off[q], true);
      cp_async_el(&sV[0][0][0] + e, a.V + base + off[q], true);
      cp_async_el(&sW[0][0][0] + e, a.W + wbase + off[q], win);
      cp_async_el(&sF[0][0][0] + e, a.phi + base + off[q], fin);
    }
    cp_async_commit();
  };
  int k = k0;
  int s_m = 0, s_0 = 0, s_p = 0;
  T g_m = T(1), g_p = T(1);   // no-slip sign of the staged u, v of planes k-1 and k+1
  const T ih = a.inv_h;
  // z-edge values of plane k at this thread's column, carried from the previous plane's
  // k+1 evaluation (the same expressions and operands, so the same values)
  T c_txz = T(0), c_tyz = T(0), c_uw = T(0), c_vw = T(0), c_tzz = T(0);
  // the faces of cell (i, j, k); SG: planes k-1 or k+1 are ghost planes beyond a z wall,
  // whose staged u, v take the no-slip sign on reading (without SG every sign is +1)
  // U >= 0: plane k sits in ring slot U (k mod 4), so every slot index is a constant;
  // U < 0: the slots of the current plane are read at run time
  auto plane = [&](auto sg_tag, auto slot_tag, size_t c, T hu, T hv, T hw, T fu, T fv, T fw) {
    constexpr bool SG = decltype(sg_tag)::value;
    constexpr int U = decltype(slot_tag)::value;
    auto pl = [&](int kk) -> int {
      if constexpr (U >= 0) return kk == k ? U : (kk > k ? ((U + 1) & (kPr - 1)) : ((U + kPr - 1) & (kPr - 1)));
      else return kk == k ? s_0 : (kk > k ? s_p : s_m);
    };
    auto sg = [&](int kk) -> T {
      if constexpr (SG) return kk == k ? T(1) : (kk > k ? g_p : g_m);
      else return T(1);
    };
    auto Cc = [&](int ii, int jj, int kk) { return sC[pl(kk)][jj - j0 + 1][ii - i0 + 1]; };
    auto Fc = [&](int ii, int jj, int kk) { return sF[pl(kk)][jj - j0 + 1][ii - i0 + 1]; };
    auto Ug = [&](int ii, int jj, int kk) {
      const T v = sU[pl(kk)][jj - j0 + 1][ii - i0 + 1];
      if constexpr (SG) return sg(kk) * v; else return v;
    };
    auto Vg = [&](int ii, int jj, int kk) {
      const T v = sV[pl(kk)][jj - j0 + 1][ii - i0 + 1];
      if constexpr (SG) return sg(kk) * v; else return v;
    };
    auto Wf = [&](int ii, int jj, int kk) { return sW[pl(kk)][jj - j0 + 1][ii - i0 + 1]; };
    auto mu = [&](T cc) { return a.mu_a + a.mu_b * clamp1(cc); };
    auto rho = [&](T cc) { return a.rho_a + a.rho_b * clamp1(cc); };
    auto txx = [&](int ii) { return T(2) * mu(Cc(ii, j, k)) * ((Ug(ii + 1, j, k) - Ug(ii, j, k)) * ih); };
    auto tyy = [&](int jj) { return T(2) * mu(Cc(i, jj, k)) * ((Vg(i, jj + 1, k) - Vg(i, jj, k)) * ih); };
    auto tzz = [&](int kk) { return T(2) * mu(Cc(i, j, kk)) * ((Wf(i, j, kk + 1) - Wf(i, j, kk)) * ih); };
    auto txy = [&](int ii, int jj, int kk) {
      const T ce = T(0.25) * (((Cc(ii - 1, jj - 1, kk) + Cc(ii, jj - 1, kk)) + Cc(ii - 1, jj, kk)) + Cc(ii, jj, kk));
      return mu(ce) * ((Ug(ii, jj, kk) - Ug(ii, jj - 1, kk)) * ih + (Vg(ii, jj, kk) - Vg(ii - 1, jj, kk)) * ih);
    };
    auto txz = [&](int ii, int jj, int kk) {
      const T ce = T(0.25) * (((Cc(ii - 1, jj, kk - 1) + Cc(ii, jj, kk - 1)) + Cc(ii - 1, jj, kk)) + Cc(ii, jj, kk));
      return mu(ce) * ((Ug(ii, jj, kk) - Ug(ii, jj, kk - 1)) * ih + (Wf(ii, jj, kk) - Wf(ii - 1, jj, kk)) * ih);
    };
    auto tyz = [&](int ii, int jj, int kk) {
      const T ce = T(0.25) * (((Cc(ii, jj - 1, kk - 1) + Cc(ii, jj, kk - 1)) + Cc(ii, jj - 1, kk)) + Cc(ii, jj, kk));
      return mu(ce) * ((Vg(ii, jj, kk) - Vg(ii, jj, kk - 1)) * ih + (Wf(ii, jj, kk) - Wf(ii, jj - 1, kk)) * ih);
    };
    auto uv = [&](int ii, int jj, int kk) {
      return (T(0.5) * (Ug(ii, jj, kk) + Ug(ii, jj - 1, kk))) * (T(0.5) * (Vg(ii, jj, kk) + Vg(ii - 1, jj, kk)));
    };
    auto uw = [&](int ii, int jj, int kk) {
      return (T(0.5) * (Ug(ii, jj, kk) + Ug(ii, jj, kk - 1))) * (T(0.5) * (Wf(ii, jj, kk) + Wf(ii - 1, jj, kk)));
    };
    auto vw = [&](int ii, int jj, int kk) {
      return (T(0.5) * (Vg(ii, jj, kk) + Vg(ii, jj, kk - 1))) * (T(0.5) * (Wf(ii, jj, kk) + Wf(ii, jj - 1, kk)));
    };
    if (k == k0) {   // first plane of the block: the k-level z-edge values directly
      c_txz = txz(i, j, k);
      c_tyz = tyz(i, j, k);
      c_uw = uw(i, j, k);
      c_vw = vw(i, j, k);
      c_tzz = tzz(k - 1);
    }
    const T n_txz = txz(i, j, k + 1), n_tyz = tyz(i, j, k + 1);
    const T n_uw = uw(i, j, k + 1), n_vw = vw(i, j, k + 1), n_tzz = tzz(k);
    const T k_st = a.k_st;
    T Hx, ux, Hy, vy, Hz = T(0), wz = T(0);
    {
      const T cL = Cc(i - 1, j, k), cR = Cc(i, j, k);
      const T rho_f = rho(T(0.5) * (cL + cR));
      const T txy0 = txy(i, j, k);
      const T visc = ((txx(i) - txx(i - 1)) * ih + (txy(i, j + 1, k) - txy0) * ih) + (n_txz - c_txz) * ih;
      const T ucR = T(0.5) * (Ug(i, j, k) + Ug(i + 1, j, k));
      const T ucL = T(0.5) * (Ug(i - 1, j, k) + Ug(i, j, k));
      const T conv = ((ucR * ucR - ucL * ucL) * ih + (uv(i, j + 1, k) - uv(i, j, k)) * ih) + (n_uw - c_uw) * ih;
      const T H = -conv + qdiv(visc, a.Re * rho_f);
      const T st = k_st * (T(0.5) * (Fc(i, j, k) + Fc(i - 1, j, k))) * qdiv((cR - cL) * ih, rho_f);
      Hx = H;
      ux = Ug(i, j, k) + a.dt * ((T(1.5) * H - T(0.5) * hu) + st);
    }
    {
      const T cB = Cc(i, j - 1, k), cA = Cc(i, j, k);
      const T rho_f = rho(T(0.5) * (cB + cA));
      const T visc = ((txy(i + 1, j, k) - txy(i, j, k)) * ih + (tyy(j) - tyy(j - 1)) * ih) + (n_tyz - c_tyz) * ih;
      const T vcA = T(0.5) * (Vg(i, j, k) + Vg(i, j + 1, k));
      const T vcB = T(0.5) * (Vg(i, j - 1, k) + Vg(i, j, k));
      const T conv = ((uv(i + 1, j, k) - uv(i, j, k)) * ih + (vcA * vcA - vcB * vcB) * ih) + (n_vw - c_vw) * ih;
      const T H = -conv + qdiv(visc, a.Re * rho_f);
      const T st = k_st * (T(0.5) * (Fc(i, j, k) + Fc(i, j - 1, k))) * qdiv((cA - cB) * ih, rho_f);
      Hy = H;
      vy = Vg(i, j, k) + a.dt * ((T(1.5) * H - T(0.5) * hv) + st);
    }
    if (k >= 1) {
      const T cB = Cc(i, j, k - 1), cA = Cc(i, j, k);
      const T rho_f = rho(T(0.5) * (cB + cA));
      const T visc = ((txz(i + 1, j, k) - c_txz) * ih + (tyz(i, j + 1, k) - c_tyz) * ih) + (n_tzz - c_tzz) * ih;
      const T wcA = T(0.5) * (Wf(i, j, k) + Wf(i, j, k + 1));
      const T wcB = T(0.5) * (Wf(i, j, k - 1) + Wf(i, j, k));
      const T conv = ((uw(i + 1, j, k) - c_uw) * ih + (vw(i, j + 1, k) - c_vw) * ih) + (wcA * wcA - wcB * wcB) * ih;
      const T H = -conv + qdiv(visc, a.Re * rho_f);
      const T st = k_st * (T(0.5) * (Fc(i, j, k) + Fc(i, j, k - 1))) * qdiv((cA - cB) * ih, rho_f);
      Hz = H;
      wz = Wf(i, j, k) + a.dt * ((T(1.5) * H - T(0.5) * hw) + st);
    }
    a.Hu[c] = Hx;
    a.Us[c] = fu * ux;
    a.Hv[c] = Hy;
    a.Vs[c] = fv * vy;
    if (k >= 1) {
      a.Hw[c] = Hz;
      a.Ws[c] = fw * wz;
    }
    c_txz = n_txz;
    c_tyz = n_tyz;
    c_uw = n_uw;
    c_vw = n_vw;
    c_tzz = n_tzz;
  };
  issue(k0 - 1);
  issue(k0);
  issue(k0 + 1);
  for (; k < k0 + kz; ++k) {
    issue(k + 2);
    const size_t c = (size_t)k * nxy + (size_t)j * a.nx + i;
    // per-face operands of plane k, requested before the wait so their latency overlaps it
    T hu = T(0), hv = T(0), hw = T(0), fu = T(0), fv = T(0), fw = T(0);
    if (active) {
      hu = a.Hu[c];
      hv = a.Hv[c];
      fu = a.au[c];
      fv = a.av[c];
      if (k >= 1) {
        hw = a.Hw[c];
        fw = a.aw[c];
      }
    }
    cp_async_wait1();   // every plane but k+2 has arrived (this thread's copies)
    __syncthreads();    // ... and every thread's
    s_m = (k + kPr - 1) & (kPr - 1);
    s_0 = k & (kPr - 1);
    s_p = (k + 1) & (kPr - 1);
    g_m = k - 1 < 0 ? T(-1) : T(1);
    g_p = k + 1 >= a.nz ? T(-1) : T(1);
    if (active) {
      using std::integral_constant;
      if (k >= 1 && k + 1 < a.nz) {
        switch (k & (kPr - 1)) {
          case 0: plane(std::false_type{}, integral_constant<int, 0>{}, c, hu, hv, hw, fu, fv, fw); break;
          case 1: plane(std::false_type{}, integral_constant<int, 1>{}, c, hu, hv, hw, fu, fv, fw); break;
          case 2: plane(std::false_type{}, integral_constant<int, 2>{}, c, hu, hv, hw, fu, fv, fw); break;
          default: plane(std::false_type{}, integral_constant<int, 3>{}, c, hu, hv, hw, fu, fv, fw); break;
        }
      } else {
        plane(std::true_type{}, integral_constant<int, -1>{}, c, hu, hv, hw, fu, fv, fw);
      }
    }
    __syncthreads();   // the slot of plane k-1 takes plane k+3 next
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");   // no copy outlives the block
}

// The FP64 form of the predictor, with the edge work shared: planes k-1, k, k+1 of C, u, v,
// w and phi staged in a four-slot ring (dynamic shared memory, k3_pred_smem bytes) filled by
// cp.async (plane k+2 in flight while plane k is computed).  Each
// thread owns the faces of cell (i, j, k) and evaluates every edge stress and product it
// needs with the same expressions as a per-face evaluation, but shares them: x-neighbour
// values (txx(i-1), txy(i+1), txz(i+1), uv(i+1), uw(i+1)) come from the adjacent lane by a
// warp shuffle (a warp is one row of 32 cells; the end lanes evaluate theirs), and the
// z-edge values of plane k+1 (txz, tyz, uw, vw at k+1 and tzz(k)) are carried in registers
// to the next plane, where they are the k-level values; the two quotients by rho_f of a
// face share one reciprocal.  The FP64 pipe, which bounds this form, does about half the
// work of the per-face evaluation.  (In the FP32 form, bound by its issue rate, the x
// shuffles measured slower; k3_predict_a carries the z values only.)
template <typename T>
__global__ void __launch_bounds__(kPx * kPy, 2) k3_predict_s(S3<T> a) {
  static_assert(kPx == 32, "one warp per tile row");
  constexpr int kSlots = kPhx * kPhy, kThreads = kPx * kPy;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* const sC = reinterpret_cast<T*>(smem_raw);
  T* const sU = sC + kPr * kSlots;
  T* const sV = sU + kPr * kSlots;
  T* const sW = sV + kPr * kSlots;
  T* const sF = sW + kPr * kSlots;
  constexpr int NS = (kSlots + kThreads - 1) / kThreads;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPx + tx;
  const int i0 = blockIdx.x * kPx, j0 = blockIdx.y * kPy;
  const int kz = a.pred_kz;
  const int k0 = blockIdx.z * kz;
  const int i = i0 + tx, j = j0 + ty;
  const bool active = i < a.nx && j < a.ny;
  const size_t nxy = (size_t)a.nx * a.ny;
  const unsigned FULL = 0xffffffffu;
  const bool first_lane = tx == 0, last_lane = tx == kPx - 1;
  // this thread's staged slots and the in-plane offsets of their columns (periodic wrap)
  unsigned off[NS];
  int sidx[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const int idx = tid + q * kThreads;
    sidx[q] = idx < kSlots ? idx : -1;
    const int r = idx / kPhx, cc = idx % kPhx;
    const int gi = (i0 - 1 + cc + a.nx) & (a.nx - 1), gj = (j0 - 1 + r + a.ny) & (a.ny - 1);
    off[q] = (unsigned)gj * (unsigned)a.nx + (unsigned)gi;
  }
  auto issue = [&](int kk) {   // plane kk (-1 .. nz+1) into slot kk mod 4
    const int sl = (kk + kPr) & (kPr - 1);
    const int km = kk < 0 ? 0 : (kk >= a.nz ? a.nz - 1 : kk);
    const bool win = kk >= 0 && kk <= a.nz, fin = kk >= 0 && kk < a.nz;
    const size_t base = (size_t)km * nxy, wbase = (size_t)(win ? kk : 0) * nxy;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      if (sidx[q] < 0) continue;
      const int e = sl * kSlots + sidx[q];
      cp_async_el(sC + e, a.C1 + base + off[q], true);
      cp_async_el(sU + e, a.U + base + off[q], true);
      cp_async_el(sV + e, a.V + base + off[q], true);
      cp_async_el(sW + e, a.W + wbase + off[q], win);
      cp_async_el(sF + e, a.phi + base + off[q], fin);
    }
    cp_async_commit();
  };
  // planes are addressed by their offset from the current plane: dk = -1, 0, +1
  int sl3[3] = {0, 0, 0};
  T sg3[3] = {T(1), T(1), T(1)};   // no-slip sign of the staged u, v (-1 beyond the z walls)
  auto at = [&](int di, int dj, int dk) { return sl3[dk + 1] * kSlots + (ty + 1 + dj) * kPhx + (tx + 1 + di); };
  auto Cc = [&](int di, int dj, int dk) { return sC[at(di, dj, dk)]; };
  auto Fc = [&](int di, int dj, int dk) { return sF[at(di, dj, dk)]; };
  auto Ug = [&](int di, int dj, int dk) { return sg3[dk + 1] * sU[at(di, dj, dk)]; };
  auto Vg = [&](int di, int dj, int dk) { return sg3[dk + 1] * sV[at(di, dj, dk)]; };
  auto Wf = [&](int di, int dj, int dk) { return sW[at(di, dj, dk)]; };
  const T ih = a.inv_h;
  const T inv_re = T(1) / a.Re;
  auto mu = [&](T cc) { return a.mu_a + a.mu_b * clamp1(cc); };
  auto rho = [&](T cc) { return a.rho_a + a.rho_b * clamp1(cc); };
  // the stresses and products, at offsets from cell (i, j, k)
  auto txx = [&](int di) { return T(2) * mu(Cc(di, 0, 0)) * ((Ug(di + 1, 0, 0) - Ug(di, 0, 0)) * ih); };
  auto tyy = [&](int dj) { return T(2) * mu(Cc(0, dj, 0)) * ((Vg(0, dj + 1, 0) - Vg(0, dj, 0)) * ih); };
  auto tzz = [&](int dk) { return T(2) * mu(Cc(0, 0, dk)) * ((Wf(0, 0, dk + 1) - Wf(0, 0, dk)) * ih); };
  auto txy = [&](int di, int dj, int dk) {
    const T ce = T(0.25) * (((Cc(di - 1, dj - 1, dk) + Cc(di, dj - 1, dk)) + Cc(di - 1, dj, dk)) + Cc(di, dj, dk));
    return mu(ce) * ((Ug(di, dj, dk) - Ug(di, dj - 1, dk)) * ih + (Vg(di, dj, dk) - Vg(di - 1, dj, dk)) * ih);
  };
  auto txz = [&](int di, int dj, int dk) {
    const T ce = T(0.25) * (((Cc(di - 1, dj, dk - 1) + Cc(di, dj, dk - 1)) + Cc(di - 1, dj, dk)) + Cc(di, dj, dk));
    return mu(ce) * ((Ug(di, dj, dk) - Ug(di, dj, dk - 1)) * ih + (Wf(di, dj, dk) - Wf(di - 1, dj, dk)) * ih);
  };
  auto tyz = [&](int di, int dj, int dk) {
    const T ce = T(0.25) * (((Cc(di, dj - 1, dk - 1) + Cc(di, dj, dk - 1)) + Cc(di, dj - 1, dk)) + Cc(di, dj, dk));
    return mu(ce) * ((Vg(di, dj, dk) - Vg(di, dj, dk - 1)) * ih + (Wf(di, dj, dk) - Wf(di, dj - 1, dk)) * ih);
  };
  auto uv = [&](int di, int dj, int dk) {
    return (T(0.5) * (Ug(di, dj, dk) + Ug(di, dj - 1, dk))) * (T(0.5) * (Vg(di, dj, dk) + Vg(di - 1, dj, dk)));
  };
  auto uw = [&](int di, int dj, int dk) {
    return (T(0.5) * (Ug(di, dj, dk) + Ug(di, dj, dk - 1))) * (T(0.5) * (Wf(di, dj, dk) + Wf(di - 1, dj, dk)));
  };
  auto vw = [&](int di, int dj, int dk) {
    return (T(0.5) * (Vg(di, dj, dk) + Vg(di, dj, dk - 1))) * (T(0.5) * (Wf(di, dj, dk) + Wf(di, dj - 1, dk)));
  };
  // z-edge values carried from the previous plane (at offsets (0,0,0) and (0,1,0) of the
  // current plane), valid after the first iteration
  T c_txz = T(0), c_tyz = T(0), c_tyzn = T(0), c_uw = T(0), c_vw = T(0), c_vwn = T(0), c_tzz = T(0);
  issue(k0 - 1);
  issue(k0);
  issue(k0 + 1);
  for (int k = k0; k < k0 + kz; ++k) {
    issue(k + 2);
    const size_t c = (size_t)k * nxy + (size_t)j * a.nx + i;
    // per-face operands of plane k, requested before the wait so their latency overlaps it
    T hu = T(0), hv = T(0), hw = T(0), fu = T(0), fv = T(0), fw = T(0);
    if (active) {
      hu = a.Hu[c];
      hv = a.Hv[c];
      fu = a.au[c];
      fv = a.av[c];
      if (k >= 1) {
        hw = a.Hw[c];
        fw = a.aw[c];
      }
    }
    cp_async_wait1();   // every plane but k+2 has arrived (this thread's copies)
    __syncthreads();    // ... and every thread's
    sl3[0] = (k + kPr - 1) & (kPr - 1);
    sl3[1] = k & (kPr - 1);
    sl3[2] = (k + 1) & (kPr - 1);
    sg3[0] = k - 1 < 0 ? T(-1) : T(1);
    sg3[2] = k + 1 >= a.nz ? T(-1) : T(1);
    if (k == k0) {   // first plane of the block: the k-level z-edge values directly
      c_txz = txz(0, 0, 0);
      c_tyz = tyz(0, 0, 0);
      c_tyzn = tyz(0, 1, 0);
      c_uw = uw(0, 0, 0);
      c_vw = vw(0, 0, 0);
      c_vwn = vw(0, 1, 0);
      c_tzz = tzz(-1);
    }
    // in-plane values with x-neighbours from the adjacent lane (every lane takes part)
    const T txx0 = txx(0);
    T txxm = __shfl_up_sync(FULL, txx0, 1);
    if (first_lane) txxm = txx(-1);
    const T txy0 = txy(0, 0, 0);
    T txyx = __shfl_down_sync(FULL, txy0, 1);
    if (last_lane) txyx = txy(1, 0, 0);
    const T uv0 = uv(0, 0, 0);
    T uvx = __shfl_down_sync(FULL, uv0, 1);
    if (last_lane) uvx = uv(1, 0, 0);
    T txzx = __shfl_down_sync(FULL, c_txz, 1);
    if (last_lane) txzx = txz(1, 0, 0);
    T uwx = __shfl_down_sync(FULL, c_uw, 1);
    if (last_lane) uwx = uw(1, 0, 0);
    // the z-edge values of plane k+1 (carried to the next iteration)
    const T n_txz = txz(0, 0, 1), n_tyz = tyz(0, 0, 1), n_tyzn = tyz(0, 1, 1);
    const T n_uw = uw(0, 0, 1), n_vw = vw(0, 0, 1), n_vwn = vw(0, 1, 1);
    const T n_tzz = tzz(0);
    if (active) {
      const T k_st = a.k_st;
      T Hx, ux, Hy, vy, Hz = T(0), wz = T(0);
      {
        const T cL = Cc(-1, 0, 0), cR = Cc(0, 0, 0);
        const T rho_f = rho(T(0.5) * (cL + cR));
        const T visc = ((txx0 - txxm) * ih + (txy(0, 1, 0) - txy0) * ih) + (n_txz - c_txz) * ih;
        const T ucR = T(0.5) * (Ug(0, 0, 0) + Ug(1, 0, 0));
        const T ucL = T(0.5) * (Ug(-1, 0, 0) + Ug(0, 0, 0));
        const T conv = ((ucR * ucR - ucL * ucL) * ih + (uv(0, 1, 0) - uv0) * ih) + (n_uw - c_uw) * ih;
        const T irho = T(1) / rho_f;   // one FP64 quotient per face
        const T H = -conv + visc * (irho * inv_re);
        const T st = k_st * (T(0.5) * (Fc(0, 0, 0) + Fc(-1, 0, 0))) * (((cR - cL) * ih) * irho);
        Hx = H;
        ux = Ug(0, 0, 0) + a.dt * ((T(1.5) * H - T(0.5) * hu) + st);
      }
      {
        const T cB = Cc(0, -1, 0), cA = Cc(0, 0, 0);
        const T rho_f = rho(T(0.5) * (cB + cA));
        const T visc = ((txyx - txy0) * ih + (tyy(0) - tyy(-1)) * ih) + (n_tyz - c_tyz) * ih;
        const T vcA = T(0.5) * (Vg(0, 0, 0) + Vg(0, 1, 0));
        const T vcB = T(0.5) * (Vg(0, -1, 0) + Vg(0, 0, 0));
        const T conv = ((uvx - uv0) * ih + (vcA * vcA - vcB * vcB) * ih) + (n_vw - c_vw) * ih;
        const T irho = T(1) / rho_f;   // one FP64 quotient per face
        const T H = -conv + visc * (irho * inv_re);
        const T st = k_st * (T(0.5) * (Fc(0, 0, 0) + Fc(0, -1, 0))) * (((cA - cB) * ih) * irho);
        Hy = H;
        vy = Vg(0, 0, 0) + a.dt * ((T(1.5) * H - T(0.5) * hv) + st);
      }
      if (k >= 1) {
        const T cB = Cc(0, 0, -1), cA = Cc(0, 0, 0);
        const T rho_f = rho(T(0.5) * (cB + cA));
        const T visc = ((txzx - c_txz) * ih + (c_tyzn - c_tyz) * ih) + (n_tzz - c_tzz) * ih;
        const T wcA = T(0.5) * (Wf(0, 0, 0) + Wf(0, 0, 1));
        const T wcB = T(0.5) * (Wf(0, 0, -1) + Wf(0, 0, 0));
        const T conv = ((uwx - c_uw) * ih + (c_vwn - c_vw) * ih) + (wcA * wcA - wcB * wcB) * ih;
        const T irho = T(1) / rho_f;   // one FP64 quotient per face
        const T H = -conv + visc * (irho * inv_re);
        const T st = k_st * (T(0.5) * (Fc(0, 0, 0) + Fc(0, 0, -1))) * (((cA - cB) * ih) * irho);
        Hz = H;
        wz = Wf(0, 0, 0) + a.dt * ((T(1.5) * H - T(0.5) * hw) + st);
      }
      a.Hu[c] = Hx;
      a.Us[c] = fu * ux;
      a.Hv[c] = Hy;
      a.Vs[c] = fv * vy;
      if (k >= 1) {
        a.Hw[c] = Hz;
        a.Ws[c] = fw * wz;
      }
    }
    c_txz = n_txz;
    c_tyz = n_tyz;
    c_tyzn = n_tyzn;
    c_uw = n_uw;
    c_vw = n_vw;
    c_vwn = n_vwn;
    c_tzz = n_tzz;
    __syncthreads();   // the slot of plane k-1 takes plane k+3 next
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");   // no copy outlives the block
}

// dynamic shared memory of k3_predict_s: five fields, four planes, the haloed tile
template <typename T>
constexpr size_t k3_pred_smem() { return sizeof(T) * 5 * kPr * kPhx * kPhy; }

// ------------------------------------------------------------- z-marching cell kernels
constexpr int kCz = 16;   // planes per block of the cell kernels
// Same blocks as the predictor: a 32 x 8 column of cells marching up kPz planes.  Fields
// differentiated in x, y or z are staged plane by plane in a rotating window with a one-cell
// halo in x and y (periodic wrap) and mirror planes beyond the z walls; each staged value is
// read from global memory once per block.
template <typename T, int NP>
struct Win {
  T p[NP][kPhy][kPhx];
};

struct Tile {
  int tx, ty, tid, i0, j0, i, j, k0, kz;
  bool active;
};

template <typename T>
__device__ __forceinline__ Tile tile3(const S3<T>& a) {
  Tile t;
  t.tx = threadIdx.x;
  t.ty = threadIdx.y;
  t.tid = t.ty * kPx + t.tx;
  t.i0 = blockIdx.x * kPx;
  t.j0 = blockIdx.y * kPy;
  t.kz = a.nz < kCz ? a.nz : kCz;
  t.k0 = blockIdx.z * t.kz;
  t.i = t.i0 + t.tx;
  t.j = t.j0 + t.ty;
  t.active = t.i < a.nx && t.j < a.ny;
  return t;
}

// stage plane kk (mirrored into 0 .. nz-1) of get(linear index) into window slot sl
template <typename T, int NP, typename G>
__device__ __forceinline__ void win_load(Win<T, NP>& w, int sl, const S3<T>& a, const Tile& t,
                                         int kk, G get) {
  const int km = kk < 0 ? 0 : (kk >= a.nz ? a.nz - 1 : kk);
  const size_t base = (size_t)km * a.nx * a.ny;
  for (int idx = t.tid; idx < kPhx * kPhy; idx += kPx * kPy) {
    const int r = idx / kPhx, q = idx % kPhx;
    const int gi = (t.i0 - 1 + q + a.nx) & (a.nx - 1), gj = (t.j0 - 1 + r + a.ny) & (a.ny - 1);
    w.p[sl][r][q] = get(base + (size_t)gj * a.nx + gi);
  }
}

__device__ __forceinline__ int slot3(int kk) { return (kk + 3) % 3; }
__device__ __forceinline__ int slot2(int kk) { return (kk + 2) & 1; }

// 7-point Laplacian from a window: (((x+ + x-) + (y+ + y-)) + (z+ + z-)) - 6 c, over h^2
template <typename T>
__device__ __forceinline__ T lap7w(const Win<T, 3>& w, int sm, int s0, int sp, const Tile& t,
                                   T inv_h2) {
  const int x = t.tx + 1, y = t.ty + 1;
  const T c0 = w.p[s0][y][x];
  return ((((w.p[s0][y][x + 1] + w.p[s0][y][x - 1]) + (w.p[s0][y + 1][x] + w.p[s0][y - 1][x])) +
           (w.p[sp][y][x] + w.p[sm][y][x])) - T(6) * c0) * inv_h2;
}

template <typename T>
__device__ __forceinline__ size_t cell_at(const S3<T>& a, const Tile& t, int k) {
  return ((size_t)k * a.ny + t.j) * a.nx + t.i;
}

// ---------------------------------------------------------------- a1: CH right-hand side
// h = (psi'(C~) - S (C~ - B))/Cn^2 - lap(B), B = C^n + (C^n - C^{n-1})/3, C~ - B = 2 d/3
template <typename T>
__global__ void __launch_bounds__(kPx * kPy) k3_ch_h_z(S3<T> a) {
  __shared__ Win<T, 3> wb, wt;
  const Tile t = tile3(a);
  const T third = T(1.0 / 3.0);
  const bool wall = a.tab.ng > 0;
  auto B = [&](size_t q) { return a.C[q] + (a.C[q] - a.Co[q]) * third; };
  auto CT = [&](size_t q) { return T(2) * a.C[q] - a.Co[q]; };
  win_load(wb, slot3(t.k0 - 1), a, t, t.k0 - 1, B);
  win_load(wb, slot3(t.k0), a, t, t.k0, B);
  if (wall) {
    win_load(wt, slot3(t.k0 - 1), a, t, t.k0 - 1, CT);
    win_load(wt, slot3(t.k0), a, t, t.k0, CT);
  }
  for (int k = t.k0; k < t.k0 + t.kz; ++k) {
    win_load(wb, slot3(k + 1), a, t, k + 1, B);
    if (wall) win_load(wt, slot3(k + 1), a, t, k + 1, CT);
    __syncthreads();
    if (t.active) {
      const size_t c = cell_at(a, t, k);
      const T lapb = lap7w(wb, slot3(k - 1), slot3(k), slot3(k + 1), t, a.inv_h2);
      const T d = a.C[c] - a.Co[c];
      const T ct = a.C[c] + d;
      a.phi[c] = ((ct * ct * ct - ct) - a.S * (T(2) * third * d)) * a.inv_eta2 - lapb;
      if (wall) {
        const T c0 = T(2) * a.C[c] - a.Co[c];
        a.rhs[c] = (c0 * c0 * c0 - c0) - a.eta2 * lap7w(wt, slot3(k - 1), slot3(k), slot3(k + 1), t, a.inv_h2);
      }
    }
    __syncthreads();
  }
}

// R = lap(h) - (Pe/Cn^2) div(u~ C~), u~ = 2u^n - u^{n-1}, C~ = 2C^n - C^{n-1}; no flux
// through the z walls
template <typename T>
__global__ void __launch_bounds__(kPx * kPy) k3_ch_rhs_z(S3<T> a) {
  __shared__ Win<T, 3> wc, wh;
  const Tile t = tile3(a);
  auto CT = [&](size_t q) { return T(2) * a.C[q] - a.Co[q]; };
  auto HH = [&](size_t q) { return a.phi[q]; };
  auto ut = [&](size_t q) { return T(2) * a.U[q] - a.Uo[q]; };
  auto vt = [&](size_t q) { return T(2) * a.V[q] - a.Vo[q]; };
  auto wt = [&](size_t q) { return T(2) * a.W[q] - a.Wo[q]; };
  const size_t nxy = (size_t)a.nx * a.ny;
  for (int kk = t.k0 - 1; kk <= t.k0; ++kk) {
    win_load(wc, slot3(kk), a, t, kk, CT);
    win_load(wh, slot3(kk), a, t, kk, HH);
  }
  const int x = t.tx + 1, y = t.ty + 1;
  for (int k = t.k0; k < t.k0 + t.kz; ++k) {
    win_load(wc, slot3(k + 1), a, t, k + 1, CT);
    win_load(wh, slot3(k + 1), a, t, k + 1, HH);
    __syncthreads();
    if (t.active) {
      const int sm = slot3(k - 1), s0 = slot3(k), sp = slot3(k + 1);
      const size_t c = cell_at(a, t, k);
      const Nbr n = nbr(a, c, t.i, t.j, k);
      const T c0 = wc.p[s0][y][x];
      const T fx_w = ut(c) * (T(0.5) * (wc.p[s0][y][x - 1] + c0));
      const T fx_e = ut(n.xp) * (T(0.5) * (c0 + wc.p[s0][y][x + 1]));
      const T fy_s = vt(c) * (T(0.5) * (wc.p[s0][y - 1][x] + c0));
      const T fy_n = vt(n.yp) * (T(0.5) * (c0 + wc.p[s0][y + 1][x]));
      const T fz_b = k > 0 ? wt(c) * (T(0.5) * (wc.p[sm][y][x] + c0)) : T(0);
      const T fz_t = k < a.nz - 1 ? wt(c + nxy) * (T(0.5) * (c0 + wc.p[sp][y][x])) : T(0);
      const T div = ((fx_e - fx_w) * a.inv_h + (fy_n - fy_s) * a.inv_h) + (fz_t - fz_b) * a.inv_h;
      a.Q[c] = lap7w(wh, sm, s0, sp, t, a.inv_h2) - a.pe_eta2 * div;
    }
    __syncthreads();
  }
}

// phi = psi'(C) - Cn^2 lap C on every cell
template <typename T>
__global__ void __launch_bounds__(kPx * kPy) k3_chem_pot_z(S3<T> a) {
  __shared__ Win<T, 3> wc;
  const Tile t = tile3(a);
  auto CC = [&](size_t q) { return a.C1[q]; };
  win_load(wc, slot3(t.k0 - 1), a, t, t.k0 - 1, CC);
  win_load(wc, slot3(t.k0), a, t, t.k0, CC);
  for (int k = t.k0; k < t.k0 + t.kz; ++k) {
    win_load(wc, slot3(k + 1), a, t, k + 1, CC);
    __syncthreads();
    if (t.active) {
      const size_t c = cell_at(a, t, k);
      const T c0 = wc.p[slot3(k)][t.ty + 1][t.tx + 1];
      a.phi[c] = (c0 * c0 * c0 - c0) - a.eta2 * lap7w(wc, slot3(k - 1), slot3(k), slot3(k + 1), t, a.inv_h2);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ a7: Poisson RHS (3D)
// lap dP = (rho0/dt) div u** - div[(rho0/rho_f) grad P^], dP = P^{n+1} - P^; stores P^
template <typename T>
__global__ void __launch_bounds__(kPx * kPy) k3_poisson_rhs_z(S3<T> a) {
  __shared__ Win<T, 3> wc, wp;
  const Tile t = tile3(a);
  auto CC = [&](size_t q) { return a.C1[q]; };
  auto PH = [&](size_t q) { return T(2) * a.P[q] - a.Po[q]; };
  auto rho = [&](T cc) { return a.rho_a + a.rho_b * clamp1(cc); };
  const size_t nxy = (size_t)a.nx * a.ny;
  for (int kk = t.k0 - 1; kk <= t.k0; ++kk) {
    win_load(wc, slot3(kk), a, t, kk, CC);
    win_load(wp, slot3(kk), a, t, kk, PH);
  }
  const int x = t.tx + 1, y = t.ty + 1;
  for (int k = t.k0; k < t.k0 + t.kz; ++k) {
    win_load(wc, slot3(k + 1), a, t, k + 1, CC);
    win_load(wp, slot3(k + 1), a, t, k + 1, PH);
    __syncthreads();
    if (t.active) {
      const int sm = slot3(k - 1), s0 = slot3(k), sp = slot3(k + 1);
      const size_t c = cell_at(a, t, k);
      const Nbr n = nbr(a, c, t.i, t.j, k);
      const T cc0 = wc.p[s0][y][x], p0 = wp.p[s0][y][x];
      const T gx_w = (a.rho0 / rho(T(0.5) * (wc.p[s0][y][x - 1] + cc0))) * ((p0 - wp.p[s0][y][x - 1]) * a.inv_h);
      const T gx_e = (a.rho0 / rho(T(0.5) * (cc0 + wc.p[s0][y][x + 1]))) * ((wp.p[s0][y][x + 1] - p0) * a.inv_h);
      const T gy_s = (a.rho0 / rho(T(0.5) * (wc.p[s0][y - 1][x] + cc0))) * ((p0 - wp.p[s0][y - 1][x]) * a.inv_h);
      const T gy_n = (a.rho0 / rho(T(0.5) * (cc0 + wc.p[s0][y + 1][x]))) * ((wp.p[s0][y + 1][x] - p0) * a.inv_h);
      T gz_b = T(0), gz_t = T(0);
      if (k > 0)
        gz_b = (a.rho0 / rho(T(0.5) * (wc.p[sm][y][x] + cc0))) * ((p0 - wp.p[sm][y][x]) * a.inv_h);
      if (k < a.nz - 1)
        gz_t = (a.rho0 / rho(T(0.5) * (cc0 + wc.p[sp][y][x]))) * ((wp.p[sp][y][x] - p0) * a.inv_h);
      const T div_g = ((gx_e - gx_w) * a.inv_h + (gy_n - gy_s) * a.inv_h) + (gz_t - gz_b) * a.inv_h;
      const T div_u = ((a.Us[n.xp] - a.Us[c]) * a.inv_h + (a.Vs[n.yp] - a.Vs[c]) * a.inv_h) +
                      (a.Ws[c + nxy] - a.Ws[c]) * a.inv_h;
      a.rhs[c] = (a.rho0 * a.inv_dt) * div_u - div_g;
      a.phat[c] = p0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------- a8: correction + status and mass (3D)
// u^{n+1} = u** - dt [ (1/rho_f) grad P^ + (1/rho0) grad dP ] on every face (z-faces 1..nz-1);
// planes k-1 and k of C, P^ and dP in two-plane windows
template <typename T>
__global__ void __launch_bounds__(kPx * kPy) k3_correct_z(S3<T> a) {
  __shared__ Win<T, 2> wc, wq, wd;
  const Tile t = tile3(a);
  auto CC = [&](size_t q) { return a.C1[q]; };
  auto PQ = [&](size_t q) { return a.phat[q]; };
  auto DP = [&](size_t q) { return a.dp[q]; };
  auto rho = [&](T cc) { return a.rho_a + a.rho_b * clamp1(cc); };
  win_load(wc, slot2(t.k0 - 1), a, t, t.k0 - 1, CC);
  win_load(wq, slot2(t.k0 - 1), a, t, t.k0 - 1, PQ);
  win_load(wd, slot2(t.k0 - 1), a, t, t.k0 - 1, DP);
  const int x = t.tx + 1, y = t.ty + 1;
  int bad = 0;
  T s_hi = T(0), s_lo = T(0);
  for (int k = t.k0; k < t.k0 + t.kz; ++k) {
    win_load(wc, slot2(k), a, t, k, CC);
    win_load(wq, slot2(k), a, t, k, PQ);
    win_load(wd, slot2(k), a, t, k, DP);
    __syncthreads();
    if (t.active) {
      const int sm = slot2(k - 1), s0 = slot2(k);
      const size_t c = cell_at(a, t, k);
      const T cc0 = wc.p[s0][y][x], q0 = wq.p[s0][y][x], d0 = wd.p[s0][y][x];
      auto corr = [&](T vel, T cnb, T qnb, T dnb) {
        const T rho_f = rho(T(0.5) * (cnb + cc0));
        const T vn = vel - a.dt * (((q0 - qnb) * a.inv_h) / rho_f + a.inv_rho0 * ((d0 - dnb) * a.inv_h));
        bad |= !isfinite(vn);
        return vn;
      };
      const T un = corr(a.Us[c], wc.p[s0][y][x - 1], wq.p[s0][y][x - 1], wd.p[s0][y][x - 1]);
      const T vn = corr(a.Vs[c], wc.p[s0][y - 1][x], wq.p[s0][y - 1][x], wd.p[s0][y - 1][x]);
      T wn = T(0);
      if (k >= 1) wn = corr(a.Ws[c], wc.p[sm][y][x], wq.p[sm][y][x], wd.p[sm][y][x]);
      bad |= !isfinite(cc0);
      a.Us[c] = un;
      a.Vs[c] = vn;
      if (k >= 1) a.Ws[c] = wn;
      pair_add(s_hi, s_lo, cc0, a.C1lo ? a.C1lo[c] : T(0));
    }
    __syncthreads();
  }
  if (bad) atomicOr(a.status, 1);
  const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int nblk = gridDim.x * gridDim.y * gridDim.z;
  tile_mass<T, kPx * kPy>(s_hi, s_lo, blk, nblk, a.partial, a.ticket, a.mass);
}

// ------------------------------------------------------------- a6: velocity ghost fill (3D)
// centred u** at the averaging cells, mirror values by Eq. extrapolation, V_nG = -V_nM/gamma
// (Eq. NoPenetration), V_tG = V_tM (l_s - dn)/(l_s + gamma dn) (Eq. UpdateVtan, static
// angle) for the tangential vector V_t = u - V_n n, u_G = V_nG n + V_tG (Eq. UpdateVandW)
template <typename T>
__device__ __forceinline__ T ucen3(const S3<T>& a, size_t c) {
  const int i = (int)(c & (size_t)(a.nx - 1));
  return T(0.5) * (a.Us[c] + a.Us[c - i + ((i + 1) & (a.nx - 1))]);
}
template <typename T>
__device__ __forceinline__ T vcen3(const S3<T>& a, size_t c) {
  const int j = (int)((c >> a.lnx) & (size_t)(a.ny - 1));
  const size_t row0 = c - ((size_t)j << a.lnx);
  return T(0.5) * (a.Vs[c] + a.Vs[row0 + ((size_t)((j + 1) & (a.ny - 1)) << a.lnx)]);
}
template <typename T>
__device__ __forceinline__ T wcen3(const S3<T>& a, size_t c) {
  return T(0.5) * (a.Ws[c] + a.Ws[c + ((size_t)a.nx << a.lny)]);
}

template <typename T>
__global__ void __launch_bounds__(kGhostBlock) k3_fill_u(S3<T> a) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int g = gt / kGhostLanes, q = gt % kGhostLanes;
  const Tables& t = a.tab;
  T s1[3], s2[3];
  gather_group<3>(t, a.w1t, a.w2t, g, q, [&](size_t c, T* v) {
    v[0] = ucen3(a, c);
    v[1] = vcen3(a, c);
    v[2] = wcen3(a, c);
  }, s1, s2);
  if (q != 0 || g >= t.ng) return;
  const T uM = T(2) * s1[0] - s2[0], vM = T(2) * s1[1] - s2[1], wM = T(2) * s1[2] - s2[2];
  const T n1 = (T)t.nrm[3 * (size_t)g], n2 = (T)t.nrm[3 * (size_t)g + 1], n3 = (T)t.nrm[3 * (size_t)g + 2];
  const T gam = (T)t.gamma[g], dn = (T)t.dn[g], ls = (T)a.l_s;
  const T vnM = (uM * n1 + vM * n2) + wM * n3;
  const T f = (ls - dn) / (ls + gam * dn);
  const T vnG = -vnM / gam;
  T gu = vnG * n1 + f * (uM - vnM * n1);
  T gv = vnG * n2 + f * (vM - vnM * n2);
  T gw = vnG * n3 + f * (wM - vnM * n3);
  if (a.a_dyn > 0.0) {
    // dynamic angle: -(1/Ca) B (dC/dx_t)_I l_s (gamma + 1) dn / (mu_I (l_s + gamma dn))
    const int ng = t.ng;
    const T mu_I = a.mu_a + a.mu_b * clamp1((T)a.ci[g]);
    const T c = (a.gq[ng + g] * (T)a.inv_ca) * (ls * (gam + T(1)) * dn) / (mu_I * (ls + gam * dn));
    gu = gu - c * a.gq[2 * ng + g];
    gv = gv - c * a.gq[3 * ng + g];
    gw = gw - c * a.gq[4 * ng + g];
  }
  a.gu[g] = gu;
  a.gv[g] = gv;
  a.gw[g] = gw;
}

// faces with alpha_f < 1 touching a ghost: mean of the two cell-centred values (ghost value,
// 0 in a solid non-ghost cell, pre-fix centred u** in a fluid cell), staged in fval
template <typename T>
__global__ void k3_face_values(S3<T> a) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const Tables& t = a.tab;
  const size_t nxy = (size_t)a.nx * a.ny;
  if (f < t.nfu) {
    const size_t c = t.fu[f];
    const int i = (int)(c & (size_t)(a.nx - 1));
    const size_t cl = c - i + ((i + a.nx - 1) & (a.nx - 1));
    auto val = [&](size_t cc) -> T {
      const int m = t.cmap[cc];
      return m >= 0 ? a.gu[m] : (m == kCellSolid ? T(0) : ucen3(a, cc));
    };
    a.fval[f] = T(0.5) * (val(cl) + val(c));
  } else if (f < t.nfu + t.nfv) {
    const size_t c = t.fv[f - t.nfu];
    const int j = (int)((c >> a.lnx) & (size_t)(a.ny - 1));
    const size_t cb = c - ((size_t)j << a.lnx) + ((size_t)((j + a.ny - 1) & (a.ny - 1)) << a.lnx);
    auto val = [&](size_t cc) -> T {
      const int m = t.cmap[cc];
      return m >= 0 ? a.gv[m] : (m == kCellSolid ? T(0) : vcen3(a, cc));
    };
    a.fval[f] = T(0.5) * (val(cb) + val(c));
  } else if (f < t.nfu + t.nfv + t.nfw) {
    const size_t c = t.fw[f - t.nfu - t.nfv];   // z-face k in 1..nz-1: cells k-1 and k
    auto val = [&](size_t cc) -> T {
      const int m = t.cmap[cc];
      return m >= 0 ? a.gw[m] : (m == kCellSolid ? T(0) : wcen3(a, cc));
    };
    a.fval[f] = T(0.5) * (val(c - nxy) + val(c));
  }
}

template <typename T>
__global__ void k3_face_scatter(S3<T> a) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const Tables& t = a.tab;
  if (f < t.nfu) a.Us[t.fu[f]] = a.fval[f];
  else if (f < t.nfu + t.nfv) a.Vs[t.fv[f - t.nfu]] = a.fval[f];
  else if (f < t.nfu + t.nfv + t.nfw) a.Ws[t.fw[f - t.nfu - t.nfv]] = a.fval[f];
}

template <typename T>
S3<T> make3(const Instance& in, int cur) {
  const ib_pf_params& p = in.prm;
  S3<T> a;
  a.nx = in.nx;
  a.ny = in.ny;
  a.nz = in.nz;
  {
    const int planes = in.tune_pred_planes ? in.tune_pred_planes : kPz;
    a.pred_kz = in.nz < planes ? in.nz : planes;
  }
  a.w1t = sizeof(T) == 8 ? (const T*)in.tab.w1 : (const T*)in.tab.w1f;
  a.w2t = sizeof(T) == 8 ? (const T*)in.tab.w2 : (const T*)in.tab.w2f;
  a.lnx = in.lognx;
  a.lny = in.logny;
  a.inv_h = (T)(1.0 / in.h);
  a.inv_h2 = (T)(1.0 / (in.h * in.h));
  a.dt = (T)p.dt;
  const double eta2 = p.Cn * p.Cn;
  a.S = (T)p.S;
  a.inv_eta2 = (T)(1.0 / eta2);
  a.pe_eta2 = (T)(p.Pe / eta2);
  a.inv_pe = (T)(1.0 / p.Pe);
  a.inv_dt = (T)(1.0 / p.dt);
  a.eta2 = (T)eta2;
  const double rho_l = 1.0, rho_g = 1.0 / p.rho_ratio, mu_l = 1.0, mu_g = 1.0 / p.mu_ratio;
  a.rho_a = (T)(0.5 * (rho_l + rho_g));
  a.rho_b = (T)(0.5 * (rho_l - rho_g));
  a.mu_a = (T)(0.5 * (mu_l + mu_g));
  a.mu_b = (T)(0.5 * (mu_l - mu_g));
  const double rho0 = rho_l < rho_g ? rho_l : rho_g;
  a.rho0 = (T)rho0;
  a.inv_rho0 = (T)(1.0 / rho0);
  a.Re = (T)p.Re;
  a.k_st = (T)(kKappa / (p.Re * p.Ca * p.Cn));
  a.k_wet = kKappa * p.Cn;
  a.cos_th = std::cos(p.theta_deg * M_PI / 180.0);
  a.l_s = p.l_s;
  a.a_dyn = p.mu_f > 0.0 ? p.dt / (p.mu_f * p.Cn) : 0.0;
  a.inv_ca = 1.0 / p.Ca;
  a.ci = (double*)in.ci;
  a.gq = (T*)in.gq;
  const int n = cur, o = 1 - cur;
  a.C = (const T*)in.C[n];
  a.Co = (const T*)in.C[o];
  a.C1 = (T*)in.C[o];
  a.C1lo = (T*)in.Clo[o];
  a.Clo = (const T*)in.Clo[n];
  a.U = (const T*)in.U[n];
  a.V = (const T*)in.V[n];
  a.W = (const T*)in.W[n];
  a.Uo = (const T*)in.U[o];
  a.Vo = (const T*)in.V[o];
  a.Wo = (const T*)in.W[o];
  a.Us = (T*)in.U[o];
  a.Vs = (T*)in.V[o];
  a.Ws = (T*)in.W[o];
  a.Hu = (T*)in.Hu;
  a.Hv = (T*)in.Hv;
  a.Hw = (T*)in.Hw;
  a.P = (const T*)in.P[n];
  a.Po = (const T*)in.P[o];
  a.Q = (T*)in.Q;
  a.phi = (T*)in.phi;
  a.rhs = (T*)in.rhs;
  a.phat = (T*)in.phat;
  a.dp = (T*)in.dp;
  a.gu = (T*)in.gu;
  a.gv = (T*)in.gv;
  a.gw = (T*)in.gw;
  a.fval = (T*)in.fval;
  if constexpr (sizeof(T) == 8) {
    a.au = (const T*)in.tab.alpha_u;
    a.av = (const T*)in.tab.alpha_v;
    a.aw = (const T*)in.tab.alpha_w;
  } else {
    const size_t cells = (size_t)in.nx * in.ny * in.nz;
    a.au = (const T*)in.alpha_f;
    a.av = (const T*)in.alpha_f + cells;
    a.aw = (const T*)in.alpha_f + 2 * cells;
  }
  a.tab = in.tab;
  a.partial = in.partial;
  a.ticket = in.ticket;
  a.mass = in.mass;
  a.status = in.status;
  return a;
}

template <typename T>
int step3d_t(const Ctx& ctx, int cur, cudaStream_t s, Recorder* rec) {
  int launches = 0;
  auto mark = [&](const char* name) {
    ++launches;
    if (rec) rec->mark(name, s);
  };
  for (const Instance& in : ctx.inst) {
    const S3<T> a = make3<T>(in, cur);
    const int ng = in.tab.ng, nf = in.tab.nfu + in.tab.nfv + in.tab.nfw;
    const unsigned gblk = (unsigned)(((size_t)ng * kGhostLanes + kGhostBlock - 1) / kGhostBlock);
    const int kzp = a.pred_kz, kzc = in.nz < kCz ? in.nz : kCz;
    const dim3 zb(kPx, kPy);
    const dim3 zg((in.nx + kPx - 1) / kPx, (in.ny + kPy - 1) / kPy, in.nz / kzc);
    const dim3 zgp((in.nx + kPx - 1) / kPx, (in.ny + kPy - 1) / kPy, in.nz / kzp);
    // FP32: four cells per thread; FP64: z-marching (each the faster form on GB300)
    const unsigned nb = (unsigned)(((size_t)in.nx * in.ny * in.nz) / (4 * kTQ));
    constexpr bool percell = sizeof(T) == 4;
    if (ctx.ch_scheme == IB_PF_CH_EXPLICIT) {
      const unsigned nbx = (unsigned)(((size_t)in.nx * in.ny * in.nz) / kTX);
      if constexpr (percell) k3x_phi2_q<<<nb, kTQ, 0, s>>>(a);
      else k3x_phi2<T><<<nbx, kTX, 0, s>>>(a);
      mark("ch_phi2");
      if (ng > 0) {
        k3x_fill2<T><<<(ng + 127) / 128, 128, 0, s>>>(a);
        mark("ch_fill2");
      }
      if constexpr (percell) k3x_update_q<<<nb, kTQ, 0, s>>>(a);
      else k3x_update<T><<<nbx, kTX, 0, s>>>(a);
      mark("ch_explicit");
    } else {
      if constexpr (percell) k3_ch_h_q<<<nb, kTQ, 0, s>>>(a);
      else k3_ch_h_z<T><<<zg, zb, 0, s>>>(a);
      mark("ch_h");
      if (ng > 0) {
        k3_ch_wall<T><<<(ng + 127) / 128, 128, 0, s>>>(a);
        mark("ch_wall");
      }
      if constexpr (percell) k3_ch_rhs_q<<<nb, kTQ, 0, s>>>(a);
      else k3_ch_rhs_z<T><<<zg, zb, 0, s>>>(a);
      mark("ch_rhs");
      launches += spectral3_solve(in, ctx.precision, 0, cur, s, rec);
    }
    if (ng > 0) {
      if (in.prm.mu_f > 0.0) {
        k3_fill_Cd<T><<<(ng + 127) / 128, 128, 0, s>>>(a, 0);
        mark("fill_C");
        k3_fill_Cd<T><<<(ng + 127) / 128, 128, 0, s>>>(a, 1);
        mark("fill_C");
      } else {
        k3_fill_C<T><<<(ng + 127) / 128, 128, 0, s>>>(a);
        mark("fill_C");
      }
    }
    if constexpr (percell) k3_chem_pot_q<<<nb, kTQ, 0, s>>>(a);
    else k3_chem_pot_z<T><<<zg, zb, 0, s>>>(a);
    mark("chem_pot");
    if (ng > 0) {
      k3_fill_phi<T><<<(ng + 127) / 128, 128, 0, s>>>(a);
      mark("fill_phi");
    }
    if constexpr (sizeof(T) == 4) k3_predict_a<T><<<zgp, zb, 0, s>>>(a);
    else k3_predict_s<T><<<zgp, zb, k3_pred_smem<T>(), s>>>(a);
    mark("predict");
    if (ng > 0) {
      k3_fill_u<T><<<gblk, kGhostBlock, 0, s>>>(a);
      mark("fill_u");
    }
    if (nf > 0) {
      k3_face_values<T><<<(nf + 127) / 128, 128, 0, s>>>(a);
      mark("face_values");
      k3_face_scatter<T><<<(nf + 127) / 128, 128, 0, s>>>(a);
      mark("face_scatter");
    }
    if constexpr (percell) k3_poisson_rhs_q<<<nb, kTQ, 0, s>>>(a);
    else k3_poisson_rhs_z<T><<<zg, zb, 0, s>>>(a);
    mark("poisson_rhs");
    launches += spectral3_solve(in, ctx.precision, 1, cur, s, rec);
    if constexpr (percell) {
      k3_correct_q<<<nb, kTQ, 0, s>>>(a);
      mark("correct");
      const int nw = (int)nb * (kTQ / 32), ngs = (nw + kMassSpan - 1) / kMassSpan;
      k3_mass_groups<<<ngs, kMassThreads, 0, s>>>(in.partial, nw, in.partial + nw);
      k3_mass_total<<<1, kMassThreads, 0, s>>>(in.partial + nw, ngs, in.mass);
      mark("mass");   // one mark for the two launches
      ++launches;
    } else {
      k3_correct_z<T><<<zg, zb, 0, s>>>(a);
      mark("correct");
    }
  }
  return launches;
}

// one launch of the 3D predictor of instance `in` with the state slot cur, writing the
// predicted velocities to us, vs, ws
template <typename T>
void predict3(const Instance& in, int cur, cudaStream_t s, void* us, void* vs, void* ws) {
  S3<T> a = make3<T>(in, cur);
  a.Us = (T*)us;
  a.Vs = (T*)vs;
  a.Ws = (T*)ws;
  const dim3 zb(kPx, kPy);
  const dim3 zgp((in.nx + kPx - 1) / kPx, (in.ny + kPy - 1) / kPy, in.nz / a.pred_kz);
  if constexpr (sizeof(T) == 4) k3_predict_a<T><<<zgp, zb, 0, s>>>(a);
  else k3_predict_s<T><<<zgp, zb, k3_pred_smem<T>(), s>>>(a);
}

}  // namespace

namespace {
__global__ void k_weights_f32(const double* __restrict__ w1, const double* __restrict__ w2,
                              float* __restrict__ f1, float* __restrict__ f2, size_t n) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    f1[e] = (float)w1[e];
    f2[e] = (float)w2[e];
  }
}
}  // namespace

// The FP32 form's ghost fills read the averaging weights in FP32: copies of the FP64 weights
// of the precompute, each rounded once (relative error 2^-24 on weights of O(1)), half the
// table bytes of every gather.
cudaError_t weights3_f32(Instance& in, cudaStream_t s) {
  const size_t n = (size_t)in.tab.ng * kNap3;
  if (in.tab.w1f) cudaFree(in.tab.w1f);
  if (in.tab.w2f) cudaFree(in.tab.w2f);
  in.tab.w1f = in.tab.w2f = nullptr;
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)&in.tab.w1f, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&in.tab.w2f, sizeof(float) * n);
  if (e != cudaSuccess) return e;
  k_weights_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in.tab.w1, in.tab.w2, in.tab.w1f, in.tab.w2f, n);
  return cudaGetLastError();
}

// Tuner: the mean time (ms) of `reps` launches of the 3D predictor of instance `in` with
// `planes` planes per block (the instance's choice is restored afterwards).  The predictor
// overwrites the AB2 history Hu, Hv, Hw, which is copied aside before and back after; its
// predicted velocities go to scratch (in a step they take the level n-1 slots, which hold
// state between steps).  -1 on a CUDA error (nothing changed).
float step3d_time_predict(const Ctx& c, Instance& in, int planes, int reps, cudaStream_t s) {
  const size_t es = c.precision == IB_PF_FP64 ? 8 : 4;
  const size_t cells = (size_t)in.nx * in.ny * in.nz, nxy = (size_t)in.nx * in.ny;
  const size_t bu = cells * es, bw = (cells + nxy) * es;
  void* save = nullptr;
  if (cudaMalloc(&save, 2 * (2 * bu + bw)) != cudaSuccess) return -1.0f;
  char* sv = (char*)save;
  cudaMemcpyAsync(sv, in.Hu, bu, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(sv + bu, in.Hv, bu, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(sv + 2 * bu, in.Hw, bw, cudaMemcpyDeviceToDevice, s);
  const int keep = in.tune_pred_planes;
  in.tune_pred_planes = planes;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto once = [&]() {
    char* out = sv + (2 * bu + bw);
    if (c.precision == IB_PF_FP64) predict3<double>(in, c.cur, s, out, out + bu, out + 2 * bu);
    else predict3<float>(in, c.cur, s, out, out + bu, out + 2 * bu);
  };
  once();   // warm-up
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) once();
  cudaEventRecord(e1, s);
  cudaMemcpyAsync(in.Hu, sv, bu, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(in.Hv, sv + bu, bu, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(in.Hw, sv + 2 * bu, bw, cudaMemcpyDeviceToDevice, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(save);
  in.tune_pred_planes = keep;
  return e == cudaSuccess ? ms / (float)reps : -1.0f;
}

int step3d(const Ctx& c, int cur, cudaStream_t s, Recorder* rec) {
  return c.precision == IB_PF_FP64 ? step3d_t<double>(c, cur, s, rec)
                                   : step3d_t<float>(c, cur, s, rec);
}

// the FP32 form reads the face fractions in FP32 (rounded once from the FP64 tables)
cudaError_t step3d_setup(Ctx& c) {
  if (c.precision == IB_PF_FP64)
    return cudaFuncSetAttribute(k3_predict_s<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)k3_pred_smem<double>());
  for (Instance& in : c.inst) {
    const size_t cells = (size_t)in.nx * in.ny * in.nz, nxy = (size_t)in.nx * in.ny;
    cudaError_t e = cudaMalloc((void**)&in.alpha_f, sizeof(float) * (3 * cells + nxy));
    if (e != cudaSuccess) return e;
    std::vector<double> hd(cells + nxy);
    std::vector<float> hf(cells + nxy);
    const double* src[3] = {in.tab.alpha_u, in.tab.alpha_v, in.tab.alpha_w};
    for (int q = 0; q < 3; ++q) {
      const size_t n = q == 2 ? cells + nxy : cells;
      e = cudaMemcpy(hd.data(), src[q], sizeof(double) * n, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return e;
      for (size_t r = 0; r < n; ++r) hf[r] = (float)hd[r];
      e = cudaMemcpy(in.alpha_f + q * cells, hf.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

}  // namespace ibpf
