// One time step of the hybrid IB / phase-field method on a 2D staggered grid
// (Sec. 4.2 and Appendix A of arXiv 2104.00350), as CUDA kernels templated on the field
// type T (double for the plain path, float for the mixed path).  Geometry tables stay FP64.
//
// Discrete operators (second-order central differences on the staggered grid, Sec. 3.1):
// cell values C, phi, P at centres; u on x1-faces (face i = left face of cell i), v on
// x2-faces (rows 0 and ny are the walls, v = 0); face values of cell quantities are
// arithmetic means; corner viscosity uses the mean C of the four surrounding cells;
// periodic in x1; at the x2 walls cell fields take mirror rows and u the no-slip ghost
// row -u.
#include <cmath>

#include <vector>

#include "batch.h"
#include "cell_common.cuh"
#include "ibpf_internal.h"

namespace ibpf {
namespace {


__device__ __forceinline__ int wrap_m(int i, int nx) { return i == 0 ? nx - 1 : i - 1; }

__device__ __forceinline__ int wrap_p(int i, int nx) { return i == nx - 1 ? 0 : i + 1; }

// cell-centred velocity components at cell c (mean of the two faces)
template <typename T>
__device__ __forceinline__ T ucen(const T* __restrict__ u, int nx, int c) {
  const int i = c % nx;
  return T(0.5) * (u[c] + u[c - i + wrap_p(i, nx)]);
}
template <typename T>
__device__ __forceinline__ T vcen(const T* __restrict__ v, int nx, int c) {
  return T(0.5) * (v[c] + v[c + nx]);
}

// ---------------------------------------------------------------- a1: CH right-hand side
// The combined solve (L^2 - (S/Cn^2) L + c0) C^{n+1} = Q of Appendix A.1, with
//   Q = (Pe/Cn^2)(C_check/dt - div(u~ C~)) + lap[(psi'(C~) - S C~)/Cn^2],  c0 = 1.5 Pe/(Cn^2 dt),
// is solved for the increment over the BDF2 predictor B = C_check / 1.5: since
// c0 B = (Pe/Cn^2) C_check/dt, the increment dC = C^{n+1} - B solves the same operator
// with right-hand side
//   R = Q - (L^2 - (S/Cn^2) L + c0) B = -(Pe/Cn^2) div(u~ C~) + lap(h),
//   h = (psi'(C~) - S (C~ - B))/Cn^2 - lap(B),
// which is small, so the solve's rounding stays relative to the change of C in one step.
// k_ch_h writes h; k_ch_rhs writes R.
// Also returns phi~ = psi'(C~) - Cn^2 lap(C~), the chemical potential of C~ that the wall term
// below fills at the ghosts (written to the rhs scratch, which the CH phase does not use).
template <typename T>
__device__ __forceinline__ T ch_h_cell(const StepArgs<T>& a, const T* __restrict__ C,
                                       const T* __restrict__ Co, int i, int j, T& phit) {
  const int nx = a.nx, ny = a.ny;
  const int im = wrap_m(i, nx), ip = wrap_p(i, nx);
  const int js = j > 0 ? j - 1 : 0, jn = j < ny - 1 ? j + 1 : ny - 1;
  const size_t r = (size_t)j * nx;
  // B = (2C^n - C^{n-1}/2)/1.5 = C^n + (C^n - C^{n-1})/3 and C~ - B = 2 (C^n - C^{n-1})/3:
  // only the small difference meets a rounded constant, so B carries no rounding bias
  const T third = T(1.0 / 3.0);
  auto bdf = [&](size_t idx) { return C[idx] + (C[idx] - Co[idx]) * third; };
  auto ctl = [&](size_t idx) { return T(2) * C[idx] - Co[idx]; };
  const T b0 = bdf(r + i);
  const size_t qn = (size_t)jn * nx + i, qs = (size_t)js * nx + i;
  const T lapb = (((bdf(r + ip) + bdf(r + im)) + (bdf(qn) + bdf(qs))) - T(4) * b0) * a.inv_h2;
  const T d = C[r + i] - Co[r + i];
  const T ct = C[r + i] + d;
  const T c0 = ctl(r + i);
  const T lapc = (((ctl(r + ip) + ctl(r + im)) + (ctl(qn) + ctl(qs))) - T(4) * c0) * a.inv_h2;
  phit = (c0 * c0 * c0 - c0) - a.eta2 * lapc;
  return ((ct * ct * ct - ct) - a.S * (T(2) * third * d)) * a.inv_eta2 - lapb;
}

template <typename T>
__device__ __forceinline__ T ch_rhs_cell(const StepArgs<T>& a, const T* __restrict__ C,
                                         const T* __restrict__ Co, const T* __restrict__ u,
                                         const T* __restrict__ uo, const T* __restrict__ v,
                                         const T* __restrict__ vo, const T* __restrict__ hf,
                                         int i, int j) {
  const int nx = a.nx, ny = a.ny;
  const int im = wrap_m(i, nx), ip = wrap_p(i, nx);
  const int js = j > 0 ? j - 1 : 0, jn = j < ny - 1 ? j + 1 : ny - 1;
  const size_t r = (size_t)j * nx;
  auto ct = [&](size_t idx) { return T(2) * C[idx] - Co[idx]; };
  const T c0 = ct(r + i), cw = ct(r + im), ce = ct(r + ip);
  const T cs = ct((size_t)js * nx + i), cn = ct((size_t)jn * nx + i);
  const T fx_w = (T(2) * u[r + i] - uo[r + i]) * (T(0.5) * (cw + c0));
  const T fx_e = (T(2) * u[r + ip] - uo[r + ip]) * (T(0.5) * (c0 + ce));
  T fy_s = T(0), fy_n = T(0);
  if (j > 0) fy_s = (T(2) * v[r + i] - vo[r + i]) * (T(0.5) * (cs + c0));
  if (j < ny - 1) fy_n = (T(2) * v[r + nx + i] - vo[r + nx + i]) * (T(0.5) * (c0 + cn));
  const T div = (fx_e - fx_w) * a.inv_h + (fy_n - fy_s) * a.inv_h;
  const T lap = (((hf[r + ip] + hf[r + im]) + (hf[(size_t)jn * nx + i] + hf[(size_t)js * nx + i])) -
                 T(4) * hf[r + i]) * a.inv_h2;
  return lap - a.pe_eta2 * div;
}

// ------------------------------------------------------------ a3: contact-angle ghost fill
// Static angle: C_M = 2 C_IP1 - C_IP2 (Eq. extrapolation) gathered with W1/W2; with G, I,
// M tied by Eq. UpdateC the normal derivative at I is (C_M - C_I)/(gamma dn), and the
// wetting condition kappa Cn dC/dn + cos(theta) g'(C_I) = 0 with g'(C) = 3/4 (1 - C^2) on
// [-1, 1] and 0 outside (the wall energy g is flat beyond the pure phases) gives:
//   |C_M| >= 1: C_I = C_M;
//   otherwise the root in [-1, 1] of a C_I^2 - k C_I + c = 0, a = -3/4 cos, c = k C_M + 3/4 cos,
//   k = kappa Cn / (gamma dn): r2 = 2c/(k + sqrt D) if |r2| <= 1, else r1 = (k + sqrt D)/(2a);
//   C_G = ((gamma + 1) C_I - C_M) / gamma   (Eq. UpdateC).
template <typename T>
__device__ __forceinline__ T gather(const T* __restrict__ f, const int* __restrict__ ap,
                                    const double* __restrict__ w, int g) {
  T acc = T(0);
#pragma unroll
  for (int q = 0; q < kNap; ++q) acc = acc + (T)w[(size_t)g * kNap + q] * f[ap[(size_t)g * kNap + q]];
  return acc;
}

template <typename T>
__device__ __forceinline__ void fill_C_ghost(const StepArgs<T>& a, const Tables& t, T* __restrict__ C,
                                             T* __restrict__ Clo, int g) {
  const T cm = T(2) * gather(C, t.ap1, t.w1, g) - gather(C, t.ap2, t.w2, g);
  const T gam = (T)t.gamma[g], dn = (T)t.dn[g];
  const T k = (T)a.k_wet / (gam * dn);
  const T qa = T(-0.75) * (T)a.cos_th;
  const T qc = k * cm + T(0.75) * (T)a.cos_th;
  T disc = k * k - T(4) * qa * qc;
  disc = disc > T(0) ? disc : T(0);
  const T sq = sqrt(disc);
  T ci = T(2) * qc / (k + sq);
  if (!(fabs(ci) <= T(1)) && qa != T(0)) {
    ci = (k + sq) / (T(2) * qa);
    ci = ci > T(1) ? T(1) : (ci < T(-1) ? T(-1) : ci);
  }
  if (fabs(cm) >= T(1)) ci = cm;
  C[t.gcell[g]] = ((gam + T(1)) * ci - cm) / gam;
  if (Clo) Clo[t.gcell[g]] = T(0);   // a ghost value is exact as stored
}

// ---------------------------------------------- a3, dynamic angle (mu_f > 0)
// Eq. WallBCS_recast for the per-ghost state C_I, one backward-Euler step in C_I:
//   F(C) = (1 + a k) C - a cos(theta) g'(C) - R = 0,  a = dt/(mu_f Cn), k = kappa Cn/(gamma dn),
//   R = C_I^n - dt v_t (dC/dx_t)_I + a k C_M,
// linear where g' = 0 (|C| >= 1): C = R/(1 + a k) if that is outside (-1, 1); otherwise the one
// root in [-1, 1] of (3/4) a cos C^2 + (1 + a k) C - (R + (3/4) a cos) = 0 (r2 = 2c/(b + sqrt D)
// if it qualifies, else r1 = -(b + sqrt D)/(2 a')).  v_t and dC/dx_t at I: gamma-weighted means
// of the ghost's value and the mirror value (Eq. interpolationAtWall) of the level-n centred
// velocity and of central differences of C^{n+1} before the fill; t = (n2, -n1).  An unset
// C_I (NaN) starts as the level-n wall value (gamma C^n_G + C^n_M)/(gamma + 1).  The results
// go to scratch (C_G, B = kappa Cn dC/dn + cos g'(C_I), dC/dx_t): no cell is written while
// other ghosts still read their neighbours.
template <typename T>
__device__ __forceinline__ void cgrad(const StepArgs<T>& a, const T* __restrict__ C, int c, T& gx,
                                      T& gy) {
  const int nx = a.nx, ny = a.ny;
  const int i = c % nx, j = c / nx;
  const int js = j > 0 ? j - 1 : 0, jn = j < ny - 1 ? j + 1 : ny - 1;
  const size_t r = (size_t)j * nx;
  const T half_inv_h = T(0.5) * a.inv_h;
  gx = (C[r + wrap_p(i, nx)] - C[r + wrap_m(i, nx)]) * half_inv_h;
  gy = (C[(size_t)jn * nx + i] - C[(size_t)js * nx + i]) * half_inv_h;
}

template <typename T>
__device__ __forceinline__ void fill_C_dynamic(const StepArgs<T>& a, const Tables& t,
                                               const T* __restrict__ C1, const T* __restrict__ Cn,
                                               const T* __restrict__ u, const T* __restrict__ v,
                                               double* __restrict__ ci, T* __restrict__ gq, int g) {
  const int nx = a.nx, ng = t.ng;
  T m1 = T(0), m2 = T(0), n1c = T(0), n2c = T(0);
  T u1 = T(0), v1 = T(0), u2 = T(0), v2 = T(0), gx1 = T(0), gy1 = T(0), gx2 = T(0), gy2 = T(0);
#pragma unroll
  for (int q = 0; q < kNap; ++q) {
    const int c1 = t.ap1[(size_t)g * kNap + q], c2 = t.ap2[(size_t)g * kNap + q];
    const T w1 = (T)t.w1[(size_t)g * kNap + q], w2 = (T)t.w2[(size_t)g * kNap + q];
    m1 = m1 + w1 * C1[c1];
    m2 = m2 + w2 * C1[c2];
    n1c = n1c + w1 * Cn[c1];
    n2c = n2c + w2 * Cn[c2];
    u1 = u1 + w1 * ucen(u, nx, c1);
    v1 = v1 + w1 * vcen(v, nx, c1);
    u2 = u2 + w2 * ucen(u, nx, c2);
    v2 = v2 + w2 * vcen(v, nx, c2);
    T gx, gy;
    cgrad(a, C1, c1, gx, gy);
    gx1 = gx1 + w1 * gx;
    gy1 = gy1 + w1 * gy;
    cgrad(a, C1, c2, gx, gy);
    gx2 = gx2 + w2 * gx;
    gy2 = gy2 + w2 * gy;
  }
  // the wall value is state that changes by a small increment every step: it is held and
  // updated in FP64 in both forms (in FP32 its rounding would accumulate like that of C)
  const int cg = t.gcell[g];
  const double gam = t.gamma[g], dn = t.dn[g];
  const double gp1 = gam + 1.0;
  const double cm = 2.0 * (double)m1 - (double)m2;
  double ci_n = ci[g];
  if (!isfinite(ci_n)) ci_n = (gam * (double)Cn[cg] + (2.0 * (double)n1c - (double)n2c)) / gp1;
  T gxg, gyg;
  cgrad(a, C1, cg, gxg, gyg);
  const T tg = (T)gam, tp1 = (T)gp1;
  const T uI = (tg * ucen(u, nx, cg) + (T(2) * u1 - u2)) / tp1;
  const T vI = (tg * vcen(v, nx, cg) + (T(2) * v1 - v2)) / tp1;
  const T gxI = (tg * gxg + (T(2) * gx1 - gx2)) / tp1;
  const T gyI = (tg * gyg + (T(2) * gy1 - gy2)) / tp1;
  const T n1 = (T)t.nrm[2 * g], n2 = (T)t.nrm[2 * g + 1];
  const T gt = gxI * n2 - gyI * n1;
  const double adv = (double)((uI * n2 - vI * n1) * gt);
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
  ci[g] = cI;
  gq[g] = (T)((gp1 * cI - cm) / gam);                                  // C_G (Eq. UpdateC)
  gq[ng + g] = (T)(k * (cm - cI) + ct * (fabs(cI) < 1.0 ? 0.75 * (1.0 - cI * cI) : 0.0));   // B
  gq[2 * ng + g] = gt;                                                 // (dC/dx_t)_I
}

// ------------------------------------------------------------- a4: chemical potential
// phi = psi'(C) - Cn^2 lap C on every cell (Eq. Chemical-Potential, nondimensional)
template <typename T>
__device__ __forceinline__ T chem_pot_cell(const StepArgs<T>& a, const T* __restrict__ C, int i,
                                           int j) {
  const int nx = a.nx, ny = a.ny;
  const size_t r = (size_t)j * nx;
  const int js = j > 0 ? j - 1 : 0, jn = j < ny - 1 ? j + 1 : ny - 1;
  const T c0 = C[r + i];
  const T lap = (((C[r + wrap_p(i, nx)] + C[r + wrap_m(i, nx)]) +
                  (C[(size_t)jn * nx + i] + C[(size_t)js * nx + i])) - T(4) * c0) * a.inv_h2;
  return (c0 * c0 * c0 - c0) - a.eta2 * lap;
}

// zero normal gradient of phi at the wall: phi_G = phi_M (Sec. 4.2.2, last paragraph)
template <typename T>
__device__ __forceinline__ void fill_phi_ghost(const Tables& t, T* __restrict__ phi, int g) {
  phi[t.gcell[g]] = T(2) * gather(phi, t.ap1, t.w1, g) - gather(phi, t.ap2, t.w2, g);
}

// ------------------------------------------- a1, wall term: no flux of C through the wall
// The explicit part of the split is lap(phi~)/Cn^2 with phi~ = psi'(C~) - Cn^2 lap(C~) the
// chemical potential of C~ = 2C^n - C^{n-1} (written by ch_h), and the wall condition
// d(phi)/dn = 0 of Eq. AllBCs is imposed on it by the ghost fill of Sec. 4.2.2,
// phi~_G = phi~_M: h at a ghost cell gains (phi~_M - phi~_G)/Cn^2.  Only ghost entries of h
// change and phi~ is read, never written, so ghosts do not read one another's results.
template <typename T>
__device__ __forceinline__ void ch_wall_ghost(const StepArgs<T>& a, const Tables& t,
                                              const T* __restrict__ phit, T* __restrict__ hf, int g) {
  const T pm = T(2) * gather(phit, t.ap1, t.w1, g) - gather(phit, t.ap2, t.w2, g);
  const int c = t.gcell[g];
  hf[c] = hf[c] + (pm - phit[c]) * a.inv_eta2;
}

// ----------------------------------------------------- a5: AB2 predictor + penalisation
// H = -div(u u) + div(mu (grad u + grad u^T)) / (Re rho_f)
// u* = u^n + dt (3/2 H^n - 1/2 H^{n-1} + (kappa/(Re Ca Cn)) phi_f dC/dx / rho_f)
// u** = alpha_f u*                                (Eqs. PredictionExp, Penalization2)
// One 32 x 8 tile per block: C, u, v and phi are staged in shared memory with a one-cell
// halo (periodic in x1; mirror rows of C and phi and no-slip ghost rows -u at the x2
// walls), then thread (i, j) updates x1-face (i, j) and, for j >= 1, x2-face (i, j).
// H is updated in place (read H^{n-1}, write H^n at the same face).
constexpr int kHx = kTileX + 2, kHy = kTileH + 2;   // staged tile with halo

template <typename T>
struct PredictSmem {
  T C[kHy][kHx];
  T U[kHy][kHx];
  T V[kHy][kHx];
  T F[kHy][kHx];   // phi
};

template <typename T>
__device__ __forceinline__ void predict_stage(const StepArgs<T>& a, const T* __restrict__ C,
                                              const T* __restrict__ phi, const T* __restrict__ u,
                                              const T* __restrict__ v, int i0, int j0,
                                              PredictSmem<T>& sm) {
  const int nx = a.nx, ny = a.ny;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int idx = tid; idx < kHx * kHy; idx += blockDim.x * blockDim.y) {
    const int r = idx / kHx, c = idx % kHx;
    const int gj = j0 - 1 + r;
    int gi = (i0 - 1 + c) % nx;
    if (gi < 0) gi += nx;
    const int cj = gj < 0 ? 0 : (gj >= ny ? ny - 1 : gj);
    sm.C[r][c] = C[(size_t)cj * nx + gi];
    sm.F[r][c] = phi[(size_t)cj * nx + gi];
    const T uu = u[(size_t)cj * nx + gi];
    sm.U[r][c] = (gj < 0 || gj >= ny) ? -uu : uu;
    sm.V[r][c] = (gj >= 0 && gj <= ny) ? v[(size_t)gj * nx + gi] : T(0);
  }
}

// (lx, ly): this cell in the staged tile; hu_old, hv_old, au, av prefetched by the caller
template <typename T>
__device__ __forceinline__ void predict_point(const StepArgs<T>& a, const PredictSmem<T>& sm,
                                              int i, int j, int lx, int ly, T hu_old, T hv_old,
                                              T au, T av, T* __restrict__ Hu,
                                              T* __restrict__ Hv, T* __restrict__ uss,
                                              T* __restrict__ vss) {
  const int nx = a.nx;
  const int tx = lx + 1, ty = ly + 1;
  const size_t r = (size_t)j * nx;
  auto Cs = [&](int di, int dj) { return sm.C[ty + dj][tx + di]; };
  auto Us = [&](int di, int dj) { return sm.U[ty + dj][tx + di]; };
  auto Vs = [&](int di, int dj) { return sm.V[ty + dj][tx + di]; };
  auto Fs = [&](int di, int dj) { return sm.F[ty + dj][tx + di]; };
  auto mu = [&](T c) { return a.mu_a + a.mu_b * clamp1(c); };
  auto rho = [&](T c) { return a.rho_a + a.rho_b * clamp1(c); };
  // corner at (i + di, j + dj) in corner indices (x = (i+di) h, y = (j+dj) h)
  auto tau_xy = [&](int di, int dj) -> T {
    const T ce = T(0.25) * (((Cs(di - 1, dj - 1) + Cs(di, dj - 1)) + Cs(di - 1, dj)) + Cs(di, dj));
    const T dudy = (Us(di, dj) - Us(di, dj - 1)) * a.inv_h;
    const T dvdx = (Vs(di, dj) - Vs(di - 1, dj)) * a.inv_h;
    return mu(ce) * (dudy + dvdx);
  };
  auto uv = [&](int di, int dj) -> T {
    return (T(0.5) * (Us(di, dj) + Us(di, dj - 1))) * (T(0.5) * (Vs(di, dj) + Vs(di - 1, dj)));
  };
  const T k_st = a.k_st;
  // ---- x1-face (i, j): cells (i-1, j) and (i, j)
  {
    const T cL = Cs(-1, 0), cR = Cs(0, 0);
    const T rho_f = rho(T(0.5) * (cL + cR));
    const T txx_R = T(2) * mu(cR) * ((Us(1, 0) - Us(0, 0)) * a.inv_h);
    const T txx_L = T(2) * mu(cL) * ((Us(0, 0) - Us(-1, 0)) * a.inv_h);
    const T visc = (txx_R - txx_L) * a.inv_h + (tau_xy(0, 1) - tau_xy(0, 0)) * a.inv_h;
    const T ucR = T(0.5) * (Us(0, 0) + Us(1, 0));
    const T ucL = T(0.5) * (Us(-1, 0) + Us(0, 0));
    const T conv = (ucR * ucR - ucL * ucL) * a.inv_h + (uv(0, 1) - uv(0, 0)) * a.inv_h;
    const T H = -conv + qdiv(visc, a.Re * rho_f);
    const T st = k_st * (T(0.5) * (Fs(0, 0) + Fs(-1, 0))) * qdiv((cR - cL) * a.inv_h, rho_f);
    const T ustar = Us(0, 0) + a.dt * ((T(1.5) * H - T(0.5) * hu_old) + st);
    Hu[r + i] = H;
    uss[r + i] = au * ustar;
  }
  // ---- x2-face (i, j), 1 <= j <= ny-1: cells (i, j-1) and (i, j)
  if (j >= 1) {
    const T cB = Cs(0, -1), cA = Cs(0, 0);
    const T rho_f = rho(T(0.5) * (cB + cA));
    const T tyy_A = T(2) * mu(cA) * ((Vs(0, 1) - Vs(0, 0)) * a.inv_h);
    const T tyy_B = T(2) * mu(cB) * ((Vs(0, 0) - Vs(0, -1)) * a.inv_h);
    const T visc = (tau_xy(1, 0) - tau_xy(0, 0)) * a.inv_h + (tyy_A - tyy_B) * a.inv_h;
    const T vcA = T(0.5) * (Vs(0, 0) + Vs(0, 1));
    const T vcB = T(0.5) * (Vs(0, -1) + Vs(0, 0));
    const T conv = (uv(1, 0) - uv(0, 0)) * a.inv_h + (vcA * vcA - vcB * vcB) * a.inv_h;
    const T H = -conv + qdiv(visc, a.Re * rho_f);
    const T st = k_st * (T(0.5) * (Fs(0, 0) + Fs(0, -1))) * qdiv((cA - cB) * a.inv_h, rho_f);
    const T vstar = Vs(0, 0) + a.dt * ((T(1.5) * H - T(0.5) * hv_old) + st);
    Hv[r + i] = H;
    vss[r + i] = av * vstar;
  }
}

// -------------------------------------- a5, semi-implicit predictor (Appendix A.2)
// Eq. predictionSemi: u* = u^n + d, (1 - (dt nu0/2) L) d = dt F with
//   F = (3/2 N^n - 1/2 N^{n-1}) + ST + V^n + MF,  N = -div(u u),  V = div(mu (grad u + grad u^T))/(Re rho_f)
// (the history field holds N only), ST the surface tension as in predict_point, and the
// mass-flux term MF = (rho'/(rho_f Pe)) (grad phi . grad) u, rho' = (rho_l - rho_g)/2: the
// chemical potential's gradient by the difference across the face and the mean of the two
// cells' central differences along it, the velocity's by central differences of its own
// faces.  This kernel writes dt F into the u** slot (the solves and the penalisation follow
// in the row / column transforms) and N into the history.
template <typename T>
__device__ __forceinline__ void predict_point_semi(const StepArgs<T>& a, const PredictSmem<T>& sm,
                                                   int i, int j, int lx, int ly, T hu_old, T hv_old,
                                                   T* __restrict__ Hu, T* __restrict__ Hv,
                                                   T* __restrict__ fu, T* __restrict__ fv) {
  const int nx = a.nx;
  const int tx = lx + 1, ty = ly + 1;
  const size_t r = (size_t)j * nx;
  auto Cs = [&](int di, int dj) { return sm.C[ty + dj][tx + di]; };
  auto Us = [&](int di, int dj) { return sm.U[ty + dj][tx + di]; };
  auto Vs = [&](int di, int dj) { return sm.V[ty + dj][tx + di]; };
  auto Fs = [&](int di, int dj) { return sm.F[ty + dj][tx + di]; };
  auto mu = [&](T c) { return a.mu_a + a.mu_b * clamp1(c); };
  auto rho = [&](T c) { return a.rho_a + a.rho_b * clamp1(c); };
  auto tau_xy = [&](int di, int dj) -> T {
    const T ce = T(0.25) * (((Cs(di - 1, dj - 1) + Cs(di, dj - 1)) + Cs(di - 1, dj)) + Cs(di, dj));
    const T dudy = (Us(di, dj) - Us(di, dj - 1)) * a.inv_h;
    const T dvdx = (Vs(di, dj) - Vs(di - 1, dj)) * a.inv_h;
    return mu(ce) * (dudy + dvdx);
  };
  auto uv = [&](int di, int dj) -> T {
    return (T(0.5) * (Us(di, dj) + Us(di, dj - 1))) * (T(0.5) * (Vs(di, dj) + Vs(di - 1, dj)));
  };
  const T k_st = a.k_st, half_ih = T(0.5) * a.inv_h, mfc = (T)a.mf_coef;
  // ---- x1-face (i, j)
  {
    const T cL = Cs(-1, 0), cR = Cs(0, 0);
    const T rho_f = rho(T(0.5) * (cL + cR));
    const T txx_R = T(2) * mu(cR) * ((Us(1, 0) - Us(0, 0)) * a.inv_h);
    const T txx_L = T(2) * mu(cL) * ((Us(0, 0) - Us(-1, 0)) * a.inv_h);
    const T visc = (txx_R - txx_L) * a.inv_h + (tau_xy(0, 1) - tau_xy(0, 0)) * a.inv_h;
    const T ucR = T(0.5) * (Us(0, 0) + Us(1, 0));
    const T ucL = T(0.5) * (Us(-1, 0) + Us(0, 0));
    const T conv = (ucR * ucR - ucL * ucL) * a.inv_h + (uv(0, 1) - uv(0, 0)) * a.inv_h;
    const T N = -conv;
    const T V = qdiv(visc, a.Re * rho_f);
    const T st = k_st * (T(0.5) * (Fs(0, 0) + Fs(-1, 0))) * qdiv((cR - cL) * a.inv_h, rho_f);
    const T phx = (Fs(0, 0) - Fs(-1, 0)) * a.inv_h;
    const T phy = T(0.5) * ((Fs(0, 1) - Fs(0, -1)) * half_ih + (Fs(-1, 1) - Fs(-1, -1)) * half_ih);
    const T ux = (Us(1, 0) - Us(-1, 0)) * half_ih, uy = (Us(0, 1) - Us(0, -1)) * half_ih;
    const T mf = qdiv(mfc, rho_f) * (phx * ux + phy * uy);
    Hu[r + i] = N;
    fu[r + i] = a.dt * ((((T(1.5) * N - T(0.5) * hu_old) + st) + V) + mf);
  }
  // ---- x2-face (i, j), 1 <= j <= ny-1; the wall faces get 0
  if (j >= 1) {
    const T cB = Cs(0, -1), cA = Cs(0, 0);
    const T rho_f = rho(T(0.5) * (cB + cA));
    const T tyy_A = T(2) * mu(cA) * ((Vs(0, 1) - Vs(0, 0)) * a.inv_h);
    const T tyy_B = T(2) * mu(cB) * ((Vs(0, 0) - Vs(0, -1)) * a.inv_h);
    const T visc = (tau_xy(1, 0) - tau_xy(0, 0)) * a.inv_h + (tyy_A - tyy_B) * a.inv_h;
    const T vcA = T(0.5) * (Vs(0, 0) + Vs(0, 1));
    const T vcB = T(0.5) * (Vs(0, -1) + Vs(0, 0));
    const T conv = (uv(1, 0) - uv(0, 0)) * a.inv_h + (vcA * vcA - vcB * vcB) * a.inv_h;
    const T N = -conv;
    const T V = qdiv(visc, a.Re * rho_f);
    const T st = k_st * (T(0.5) * (Fs(0, 0) + Fs(0, -1))) * qdiv((cA - cB) * a.inv_h, rho_f);
    const T phx = T(0.5) * ((Fs(1, 0) - Fs(-1, 0)) * half_ih + (Fs(1, -1) - Fs(-1, -1)) * half_ih);
    const T phy = (Fs(0, 0) - Fs(0, -1)) * a.inv_h;
    const T vx = (Vs(1, 0) - Vs(-1, 0)) * half_ih, vy = (Vs(0, 1) - Vs(0, -1)) * half_ih;
    const T mf = qdiv(mfc, rho_f) * (phx * vx + phy * vy);
    Hv[r + i] = N;
    fv[r + i] = a.dt * ((((T(1.5) * N - T(0.5) * hv_old) + st) + V) + mf);
  } else {
    fv[r + i] = T(0);
  }
}

// ------------------------------------------------------------- a6: velocity ghost fill
// centred u** at the averaging points, mirror value by Eq. extrapolation, then
// V_nG = -V_nM / gamma (Eq. NoPenetration), V_tG = V_tM (l_s - dn)/(l_s + gamma dn)
// (Eq. UpdateVtan with the static-angle bracket zero), t = (n2, -n1), Eq. UpdateVandW.

template <typename T>
__device__ __forceinline__ void fill_u_ghost(const StepArgs<T>& a, const Tables& t,
                                             const T* __restrict__ uss, const T* __restrict__ vss,
                                             T* __restrict__ gu, T* __restrict__ gv,
                                             const double* __restrict__ ci, const T* __restrict__ gq,
                                             int g) {
  const int nx = a.nx;
  T u1 = T(0), v1 = T(0), u2 = T(0), v2 = T(0);
#pragma unroll
  for (int q = 0; q < kNap; ++q) {
    const int c1 = t.ap1[(size_t)g * kNap + q], c2 = t.ap2[(size_t)g * kNap + q];
    const T w1 = (T)t.w1[(size_t)g * kNap + q], w2 = (T)t.w2[(size_t)g * kNap + q];
    u1 = u1 + w1 * ucen(uss, nx, c1);
    v1 = v1 + w1 * vcen(vss, nx, c1);
    u2 = u2 + w2 * ucen(uss, nx, c2);
    v2 = v2 + w2 * vcen(vss, nx, c2);
  }
  const T uM = T(2) * u1 - u2, vM = T(2) * v1 - v2;
  const T n1 = (T)t.nrm[2 * g], n2 = (T)t.nrm[2 * g + 1];
  const T gam = (T)t.gamma[g], dn = (T)t.dn[g], ls = (T)a.l_s;
  const T vnM = uM * n1 + vM * n2;
  const T vtM = uM * n2 - vM * n1;
  const T vnG = -vnM / gam;
  T vtG = vtM * (ls - dn) / (ls + gam * dn);
  if (a.a_dyn > 0.0) {
    // dynamic angle: -(1/Ca) B (dC/dx_t)_I l_s (gamma + 1) dn / (mu_I (l_s + gamma dn))
    const int ng = t.ng;
    const T mu_I = a.mu_a + a.mu_b * clamp1((T)ci[g]);
    vtG = vtG - (gq[ng + g] * gq[2 * ng + g] * (T)a.inv_ca) * (ls * (gam + T(1)) * dn) /
                    (mu_I * (ls + gam * dn));
  }
  gu[g] = vnG * n1 + vtG * n2;
  gv[g] = vnG * n2 - vtG * n1;
}

// faces with alpha_f < 1 touching a ghost: mean of the two cell-centred values (ghost
// value, 0 in a solid non-ghost cell, pre-fix centred u** in a fluid cell).  Values go to
// fval first so that no face is overwritten while a neighbour still reads it.
template <typename T>
__device__ __forceinline__ void face_value(const StepArgs<T>& a, const Tables& t,
                                           const T* __restrict__ uss, const T* __restrict__ vss,
                                           const T* __restrict__ gu, const T* __restrict__ gv,
                                           T* __restrict__ fval, int f) {
  const int nx = a.nx;
  if (f < t.nfu) {
    const int c = t.fu[f];
    const int i = c % nx;
    const int cl = c - i + wrap_m(i, nx);
    auto val = [&](int cc) -> T {
      const int m = t.cmap[cc];
      return m >= 0 ? gu[m] : (m == kCellSolid ? T(0) : ucen(uss, nx, cc));
    };
    fval[f] = T(0.5) * (val(cl) + val(c));
  } else if (f < t.nfu + t.nfv) {
    const int c = t.fv[f - t.nfu];
    const int cb = c - nx;
    auto val = [&](int cc) -> T {
      const int m = t.cmap[cc];
      return m >= 0 ? gv[m] : (m == kCellSolid ? T(0) : vcen(vss, nx, cc));
    };
    fval[f] = T(0.5) * (val(cb) + val(c));
  }
}

template <typename T>
__device__ __forceinline__ void face_scatter(const Tables& t, const T* __restrict__ fval,
                                             T* __restrict__ uss, T* __restrict__ vss, int f) {
  if (f < t.nfu) uss[t.fu[f]] = fval[f];
  else if (f < t.nfu + t.nfv) vss[t.fv[f - t.nfu]] = fval[f];
}

// ------------------------------------------------------------------ a7: Poisson RHS
// Eq. PressurePoisson, lap P^{n+1} = div[(1 - rho0/rho_f) grad P^] + (rho0/dt) div u**,
// P^ = 2P^n - P^{n-1}, solved for the increment dP = P^{n+1} - P^:
//   lap dP = (rho0/dt) div u** - div[(rho0/rho_f) grad P^]     (zero flux at the x2 walls).
// Also stores P^ for the correction.
template <typename T>
__device__ __forceinline__ void poisson_rhs_cell(const StepArgs<T>& a, const T* __restrict__ C,
                                                 const T* __restrict__ P, const T* __restrict__ Po,
                                                 const T* __restrict__ uss, const T* __restrict__ vss,
                                                 T& rhs, T& phat, int i, int j) {
  const int nx = a.nx, ny = a.ny;
  const int im = wrap_m(i, nx), ip = wrap_p(i, nx);
  const size_t r = (size_t)j * nx;
  auto ph = [&](size_t idx) { return T(2) * P[idx] - Po[idx]; };
  auto rho = [&](T c) { return a.rho_a + a.rho_b * clamp1(c); };
  const T p0 = ph(r + i);
  const T gx_w = (a.rho0 / rho(T(0.5) * (C[r + im] + C[r + i]))) * ((p0 - ph(r + im)) * a.inv_h);
  const T gx_e = (a.rho0 / rho(T(0.5) * (C[r + i] + C[r + ip]))) * ((ph(r + ip) - p0) * a.inv_h);
  T gy_s = T(0), gy_n = T(0);
  if (j > 0)
    gy_s = (a.rho0 / rho(T(0.5) * (C[r - nx + i] + C[r + i]))) * ((p0 - ph(r - nx + i)) * a.inv_h);
  if (j < ny - 1)
    gy_n = (a.rho0 / rho(T(0.5) * (C[r + i] + C[r + nx + i]))) * ((ph(r + nx + i) - p0) * a.inv_h);
  const T div_g = (gx_e - gx_w) * a.inv_h + (gy_n - gy_s) * a.inv_h;
  const T div_u = (uss[r + ip] - uss[r + i]) * a.inv_h + (vss[r + nx + i] - vss[r + i]) * a.inv_h;
  rhs = (a.rho0 * a.inv_dt) * div_u - div_g;
  phat = p0;
}

// ------------------------------------------------- a8: correction + status and mass
// Eq. correction, u^{n+1} = u** - dt [ (1/rho0) grad P^{n+1} + (1/rho_f - 1/rho0) grad P^ ],
// written with the increment: u^{n+1} = u** - dt [ (1/rho_f) grad P^ + (1/rho0) grad dP ].
// Returns u^{n+1} (and v^{n+1} for j >= 1) of this cell's faces; flags non-finite values.
template <typename T>
__device__ __forceinline__ void correct_cell(const StepArgs<T>& a, const T* __restrict__ C,
                                             const T* __restrict__ dP, const T* __restrict__ phat,
                                             const T* __restrict__ uss, const T* __restrict__ vss,
                                             int i, int j, T& un, T& vn, int& bad) {
  const int nx = a.nx;
  const int im = wrap_m(i, nx);
  const size_t r = (size_t)j * nx;
  auto rho = [&](T c) { return a.rho_a + a.rho_b * clamp1(c); };
  {
    const T rho_f = rho(T(0.5) * (C[r + im] + C[r + i]));
    un = uss[r + i] - a.dt * (((phat[r + i] - phat[r + im]) * a.inv_h) / rho_f +
                              a.inv_rho0 * ((dP[r + i] - dP[r + im]) * a.inv_h));
    bad |= !isfinite(un);
  }
  if (j >= 1) {
    const size_t rs = r - nx;
    const T rho_f = rho(T(0.5) * (C[rs + i] + C[r + i]));
    vn = vss[r + i] - a.dt * (((phat[r + i] - phat[rs + i]) * a.inv_h) / rho_f +
                              a.inv_rho0 * ((dP[r + i] - dP[rs + i]) * a.inv_h));
    bad |= !isfinite(vn);
  }
  bad |= !isfinite(C[r + i]);
}

// stand-alone FP64 sum of a cell field (same reduction as in k_correct)
template <typename T>
__global__ void k_mass(int n, const T* __restrict__ C, const T* __restrict__ Clo,
                       double* __restrict__ partial,
                       unsigned* __restrict__ ticket, double* __restrict__ mass) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  double csum = 0.0;
  for (int k = blockIdx.x * nthr + tid; k < n; k += gridDim.x * nthr)
    csum += (double)C[k] + (Clo ? (double)Clo[k] : 0.0);
  __shared__ double red[256];
  red[tid] = csum;
  __syncthreads();
  for (int s = nthr / 2; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  __shared__ bool last;
  if (tid == 0) {
    partial[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (unsigned b = tid; b < gridDim.x; b += nthr) s += ((volatile double*)partial)[b];
    red[tid] = s;
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
}

template <typename T>
StepArgs<T> make_args(const Instance& in) {
  const ib_pf_params& p = in.prm;
  StepArgs<T> a;
  a.nx = in.nx;
  a.ny = in.ny;
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
  a.mf_coef = 0.5 * (rho_l - rho_g) / p.Pe;
  return a;
}

// ------------------------------------------------------------ batched launches
// Block b of a launch takes entry b of its family's block table: (instance, block within
// the instance).  Cell tiles are 32 x 32 cells (32 x 8 threads, 4 rows each); ghost and face
// families use chunks of 128.

#define IBPF_CELL_BOUNDS __launch_bounds__(kTileX * kTileY)

// first cell of this thread in tile lb: column i, rows jb, jb + 8, jb + 16, jb + 24
template <typename T>
__device__ __forceinline__ void tile_base(const InstDev<T>& d, int lb, int& i, int& jb) {
  i = (lb % d.gx) * kTileX + threadIdx.x;
  jb = (lb / d.gx) * kTileH + threadIdx.y;
}

template <typename T>
__global__ void IBPF_CELL_BOUNDS kb_ch_h(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk, int nblk,
                        int cur) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    int i, jb;
    tile_base(d, w_.y, i, jb);
    // all rows are computed before any is stored, so that the loads of every row are in
    // flight together (a store could alias a later row's loads as far as the compiler knows)
    T out[kRowsPerThread], pt[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny) out[q] = ch_h_cell(d.a, d.C[cur], d.C[1 - cur], i, j, pt[q]);
    }
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny) {
        d.phi[(size_t)j * d.nx + i] = out[q];
        if (d.tab.ng > 0) d.rhs[(size_t)j * d.nx + i] = pt[q];
      }
    }
  }
}

template <typename T>
__global__ void IBPF_CELL_BOUNDS kb_ch_rhs(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk, int nblk,
                          int cur) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    int i, jb;
    tile_base(d, w_.y, i, jb);
    T out[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny)
        out[q] = ch_rhs_cell(d.a, d.C[cur], d.C[1 - cur], d.U[cur], d.U[1 - cur], d.V[cur],
                             d.V[1 - cur], d.phi, i, j);
    }
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny) d.Q[(size_t)j * d.nx + i] = out[q];
    }
  }
}

template <typename T>
__global__ void kb_ch_wall(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk, int nblk,
                           int cur) {
  const int b_ = blockIdx.x;
  if (b_ >= nblk) return;
  const int2 w_ = blk[b_];
  const InstDev<T>& d = I[w_.x];
  const int g = w_.y * kGhostChunk + threadIdx.x;
  if (g < d.tab.ng) ch_wall_ghost(d.a, d.tab, d.rhs, d.phi, g);
}

// C^{n+1} sits in slot 1 - cur after the CH solve.  Static angle: one pass.  Dynamic angle
// (instances with mu_f > 0): pass 0 computes into scratch, pass 1 writes the ghost cells.
template <typename T>
__global__ void kb_fill_C(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk, int nblk,
                          int cur, int pass) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    const int g = w_.y * kGhostChunk + threadIdx.x;
    if (g >= d.tab.ng) return;
    if (d.a.a_dyn > 0.0) {
      if (pass == 0) {
        fill_C_dynamic(d.a, d.tab, d.C[1 - cur], d.C[cur], d.U[cur], d.V[cur], d.ci, d.gq, g);
      } else {
        d.C[1 - cur][d.tab.gcell[g]] = d.gq[g];
        if (d.Clo[1 - cur]) d.Clo[1 - cur][d.tab.gcell[g]] = T(0);
      }
    } else if (pass == 0) {
      fill_C_ghost(d.a, d.tab, d.C[1 - cur], d.Clo[1 - cur], g);
    }
  }
}

template <typename T>
__global__ void IBPF_CELL_BOUNDS kb_chem_pot(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                            int nblk, int cur) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    int i, jb;
    tile_base(d, w_.y, i, jb);
    T out[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny) out[q] = chem_pot_cell(d.a, d.C[1 - cur], i, j);
    }
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny) d.phi[(size_t)j * d.nx + i] = out[q];
    }
  }
}

template <typename T>
__global__ void kb_fill_phi(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                            int nblk) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    const int g = w_.y * kGhostChunk + threadIdx.x;
    if (g < d.tab.ng) fill_phi_ghost(d.tab, d.phi, g);
  }
}

// u** goes into the u^{n-1} slot (1 - cur); SEMI: dt F of the semi-implicit predictor
template <typename T, bool SEMI>
__global__ void IBPF_CELL_BOUNDS kb_predict(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                           int nblk, int cur) {
  __shared__ PredictSmem<T> sm;
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    const int i0 = (w_.y % d.gx) * kTileX, j0 = (w_.y / d.gx) * kTileH;
    const int i = i0 + threadIdx.x;
    // own-face history and penalisation factors, fetched while the tile is staged
    T huo[kRowsPerThread], hvo[kRowsPerThread];
    T au[kRowsPerThread], av[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = j0 + threadIdx.y + q * kTileY;
      const bool ok = i < d.nx && j < d.ny;
      const size_t c = (size_t)j * d.nx + i;
      huo[q] = ok ? d.Hu[c] : T(0);
      hvo[q] = ok ? d.Hv[c] : T(0);
      au[q] = ok ? d.au[c] : T(0);
      av[q] = ok ? d.av[c] : T(0);
    }
    predict_stage(d.a, d.C[1 - cur], d.phi, d.U[cur], d.V[cur], i0, j0, sm);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int ly = threadIdx.y + q * kTileY;
      const int j = j0 + ly;
      if (i < d.nx && j < d.ny) {
        if constexpr (SEMI)
          predict_point_semi(d.a, sm, i, j, threadIdx.x, ly, huo[q], hvo[q], d.Hu, d.Hv,
                             d.U[1 - cur], d.V[1 - cur]);
        else
          predict_point(d.a, sm, i, j, threadIdx.x, ly, huo[q], hvo[q], au[q], av[q], d.Hu, d.Hv,
                        d.U[1 - cur], d.V[1 - cur]);
      }
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void kb_fill_u(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk, int nblk,
                          int cur) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    const int g = w_.y * kGhostChunk + threadIdx.x;
    if (g < d.tab.ng) fill_u_ghost(d.a, d.tab, d.U[1 - cur], d.V[1 - cur], d.gu, d.gv, d.ci, d.gq, g);
  }
}

template <typename T>
__global__ void kb_face_values(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                               int nblk, int cur) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    const int f = w_.y * kGhostChunk + threadIdx.x;
    face_value(d.a, d.tab, d.U[1 - cur], d.V[1 - cur], d.gu, d.gv, d.fval, f);
  }
}

template <typename T>
__global__ void kb_face_scatter(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                                int nblk, int cur) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    const int f = w_.y * kGhostChunk + threadIdx.x;
    face_scatter(d.tab, d.fval, d.U[1 - cur], d.V[1 - cur], f);
  }
}

template <typename T>
__global__ void IBPF_CELL_BOUNDS kb_poisson_rhs(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                               int nblk, int cur) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    int i, jb;
    tile_base(d, w_.y, i, jb);
    T o_rhs[kRowsPerThread], o_ph[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny)
        poisson_rhs_cell(d.a, d.C[1 - cur], d.P[cur], d.P[1 - cur], d.U[1 - cur], d.V[1 - cur],
                         o_rhs[q], o_ph[q], i, j);
    }
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny) {
        d.rhs[(size_t)j * d.nx + i] = o_rhs[q];
        d.phat[(size_t)j * d.nx + i] = o_ph[q];
      }
    }
  }
}

template <typename T>
__global__ void IBPF_CELL_BOUNDS kb_correct(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                           int nblk, int cur) {
  {   // one block per work unit (the grid is nblk blocks)
    const int b_ = blockIdx.x;
    if (b_ >= nblk) return;
    const int2 w_ = blk[b_];
    const InstDev<T>& d = I[w_.x];
    int i, jb, bad = 0;
    tile_base(d, w_.y, i, jb);
    T s_hi = T(0), s_lo = T(0);
    T o_u[kRowsPerThread], o_v[kRowsPerThread];
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny) {
        correct_cell(d.a, d.C[1 - cur], d.dp, d.phat, d.U[1 - cur], d.V[1 - cur], i, j, o_u[q],
                     o_v[q], bad);
        const size_t c = (size_t)j * d.nx + i;
        const T lo = d.Clo[1 - cur] ? d.Clo[1 - cur][c] : T(0);
        pair_add(s_hi, s_lo, d.C[1 - cur][c], lo);
      }
    }
#pragma unroll
    for (int q = 0; q < kRowsPerThread; ++q) {
      const int j = jb + q * kTileY;
      if (i < d.nx && j < d.ny) {
        d.U[1 - cur][(size_t)j * d.nx + i] = o_u[q];
        if (j >= 1) d.V[1 - cur][(size_t)j * d.nx + i] = o_v[q];
      }
    }
    if (bad) atomicOr(d.status, 1);
    const int ntiles = d.gx * ((d.ny + kTileH - 1) / kTileH);
    tile_mass<T, kTileX * kTileY>(s_hi, s_lo, w_.y, ntiles, d.partial, d.ticket, d.mass);
  }
}

// ------------------------------------------- FP32 form: four cells per thread
// The same 32 x 32 cell tiles and block tables, each thread owning a run of four
// x1-consecutive cells of one row (8 runs x 32 rows; a warp holds 4 row segments of 8 runs).
// One 16-byte load per field and row; the x1 neighbours of a run come from the adjacent
// lanes by shuffles.  The arithmetic of each cell is that of the *_cell functions above, term
// for term.  Threads of a partial tile (nx or ny below 32) take part in the shuffles with
// loads of cell 0 and store nothing.
struct Run2 {
  size_t q, s, n, xl, xr;   // first cell of the run, the runs below / above (mirror), x wrap
  int i0, j, gl;
  bool act;
};
__device__ __forceinline__ Run2 run2(const InstDev<float>& d, int lb) {
  Run2 r;
  const int tid = threadIdx.y * kTileX + threadIdx.x;
  r.gl = tid & 7;
  const int i0 = (lb % d.gx) * kTileX + 4 * r.gl, j = (lb / d.gx) * kTileH + (tid >> 3);
  const int nx = d.nx, ny = d.ny;
  r.act = i0 < nx && j < ny;
  r.i0 = r.act ? i0 : 0;
  r.j = r.act ? j : 0;
  r.q = (size_t)r.j * nx + r.i0;
  r.s = (size_t)(r.j > 0 ? r.j - 1 : 0) * nx + r.i0;
  r.n = (size_t)(r.j < ny - 1 ? r.j + 1 : ny - 1) * nx + r.i0;
  r.xl = r.i0 == 0 ? r.q + (nx - 1) : r.q - 1;
  r.xr = r.i0 + 4 == nx ? r.q + 4 - nx : r.q + 4;
  return r;
}
template <typename G>
__device__ __forceinline__ X2 xnb2(const V4& v, const Run2& r, int nx, G get) {
  return xnb<8>(v, r.gl, r.i0 == 0, r.i0 + 4 == nx, r.xl, r.xr, get);
}

// 5-point Laplacian of cell e of a run (xp + xm first, as the *_cell functions)
__device__ __forceinline__ float lap5q(const StepArgs<float>& a, const V4& c, const X2& x,
                                       const V4& n, const V4& s, int e) {
  return (((right(c, x, e) + left(c, x, e)) + (n.e[e] + s.e[e])) - 4.0f * c.e[e]) * a.inv_h2;
}

#define IBPF_QUAD_PROLOGUE                 \
  const int b_ = blockIdx.x;               \
  if (b_ >= nblk) return;                  \
  const int2 w_ = blk[b_];                 \
  const InstDev<float>& d = I[w_.x];       \
  const StepArgs<float>& a = d.a;          \
  const Run2 r = run2(d, w_.y);

__global__ void IBPF_CELL_BOUNDS kq_ch_h(const InstDev<float>* __restrict__ I, const int2* __restrict__ blk,
                                         int nblk, int cur) {
  IBPF_QUAD_PROLOGUE
  const float* C = d.C[cur];
  const float* Co = d.C[1 - cur];
  const float third = float(1.0 / 3.0);
  auto B4 = [&](size_t q) {
    const V4 c = ld4(C, q), o = ld4(Co, q);
    return map4([&](int e) { return c.e[e] + (c.e[e] - o.e[e]) * third; });
  };
  const V4 c = ld4(C, r.q), o = ld4(Co, r.q);
  const V4 b = map4([&](int e) { return c.e[e] + (c.e[e] - o.e[e]) * third; });
  const V4 bn = B4(r.n), bs = B4(r.s);
  const X2 bx = xnb2(b, r, d.nx, [&](size_t q) { return C[q] + (C[q] - Co[q]) * third; });
  const V4 out = map4([&](int e) {
    const float dd = c.e[e] - o.e[e];
    const float ct = c.e[e] + dd;
    return ((ct * ct * ct - ct) - a.S * (2.0f * third * dd)) * a.inv_eta2 - lap5q(a, b, bx, bn, bs, e);
  });
  if (r.act) st4(d.phi, r.q, out);
  if (d.tab.ng > 0) {
    // phi~ = psi'(C~) - Cn^2 lap(C~) for the wall term (ch_wall), into the rhs scratch
    auto T4 = [&](size_t q) {
      const V4 x = ld4(C, q), y = ld4(Co, q);
      return map4([&](int e) { return 2.0f * x.e[e] - y.e[e]; });
    };
    const V4 ct = map4([&](int e) { return 2.0f * c.e[e] - o.e[e]; });
    const V4 tn = T4(r.n), ts = T4(r.s);
    const X2 tx = xnb2(ct, r, d.nx, [&](size_t q) { return 2.0f * C[q] - Co[q]; });
    const V4 pt = map4([&](int e) {
      const float x = ct.e[e];
      return (x * x * x - x) - a.eta2 * lap5q(a, ct, tx, tn, ts, e);
    });
    if (r.act) st4(d.rhs, r.q, pt);
  }
}

__global__ void IBPF_CELL_BOUNDS kq_ch_rhs(const InstDev<float>* __restrict__ I, const int2* __restrict__ blk,
                                           int nblk, int cur) {
  IBPF_QUAD_PROLOGUE
  const float *C = d.C[cur], *Co = d.C[1 - cur], *u = d.U[cur], *uo = d.U[1 - cur];
  const float *v = d.V[cur], *vo = d.V[1 - cur], *hf = d.phi;
  const int nx = d.nx, ny = d.ny;
  auto two = [&](const float* f, const float* fo, size_t q) {
    const V4 x = ld4(f, q), y = ld4(fo, q);
    return map4([&](int e) { return 2.0f * x.e[e] - y.e[e]; });
  };
  const V4 c0 = two(C, Co, r.q), cn = two(C, Co, r.n), cs = two(C, Co, r.s);
  const V4 ut = two(u, uo, r.q), vt = two(v, vo, r.q), vtn = two(v, vo, r.q + nx);
  const V4 h = ld4(hf, r.q), hn = ld4(hf, r.n), hs = ld4(hf, r.s);
  const X2 cx = xnb2(c0, r, nx, [&](size_t q) { return 2.0f * C[q] - Co[q]; });
  const X2 ux = xnb2(ut, r, nx, [&](size_t q) { return 2.0f * u[q] - uo[q]; });
  const X2 hx = xnb2(h, r, nx, [&](size_t q) { return hf[q]; });
  const V4 out = map4([&](int e) {
    const float cc = c0.e[e];
    const float fx_w = ut.e[e] * (0.5f * (left(c0, cx, e) + cc));
    const float fx_e = right(ut, ux, e) * (0.5f * (cc + right(c0, cx, e)));
    float fy_s = 0.0f, fy_n = 0.0f;
    if (r.j > 0) fy_s = vt.e[e] * (0.5f * (cs.e[e] + cc));
    if (r.j < ny - 1) fy_n = vtn.e[e] * (0.5f * (cc + cn.e[e]));
    const float div = (fx_e - fx_w) * a.inv_h + (fy_n - fy_s) * a.inv_h;
    return lap5q(a, h, hx, hn, hs, e) - a.pe_eta2 * div;
  });
  if (r.act) st4(d.Q, r.q, out);
}

__global__ void IBPF_CELL_BOUNDS kq_chem_pot(const InstDev<float>* __restrict__ I, const int2* __restrict__ blk,
                                             int nblk, int cur) {
  IBPF_QUAD_PROLOGUE
  const float* C = d.C[1 - cur];
  const V4 c = ld4(C, r.q), cn = ld4(C, r.n), cs = ld4(C, r.s);
  const X2 cx = xnb2(c, r, d.nx, [&](size_t q) { return C[q]; });
  const V4 out = map4([&](int e) {
    const float c0 = c.e[e];
    return (c0 * c0 * c0 - c0) - a.eta2 * lap5q(a, c, cx, cn, cs, e);
  });
  if (r.act) st4(d.phi, r.q, out);
}

__global__ void IBPF_CELL_BOUNDS kq_poisson_rhs(const InstDev<float>* __restrict__ I,
                                                const int2* __restrict__ blk, int nblk, int cur) {
  IBPF_QUAD_PROLOGUE
  const float *C = d.C[1 - cur], *P = d.P[cur], *Po = d.P[1 - cur];
  const float *uss = d.U[1 - cur], *vss = d.V[1 - cur];
  const int nx = d.nx, ny = d.ny;
  auto rho = [&](float cc) { return a.rho_a + a.rho_b * clamp1(cc); };
  auto ph4 = [&](size_t q) {
    const V4 p = ld4(P, q), po = ld4(Po, q);
    return map4([&](int e) { return 2.0f * p.e[e] - po.e[e]; });
  };
  const V4 p0 = ph4(r.q), pn = ph4(r.n), ps = ph4(r.s);
  const V4 c0 = ld4(C, r.q), cn = ld4(C, r.n), cs = ld4(C, r.s);
  const V4 us = ld4(uss, r.q), vs = ld4(vss, r.q), vsn = ld4(vss, r.q + nx);
  const X2 px = xnb2(p0, r, nx, [&](size_t q) { return 2.0f * P[q] - Po[q]; });
  const X2 cx = xnb2(c0, r, nx, [&](size_t q) { return C[q]; });
  const X2 ux = xnb2(us, r, nx, [&](size_t q) { return uss[q]; });
  V4 rhs;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float pc = p0.e[e], cc = c0.e[e];
    const float gx_w = qdiv(a.rho0, rho(0.5f * (left(c0, cx, e) + cc))) * ((pc - left(p0, px, e)) * a.inv_h);
    const float gx_e = qdiv(a.rho0, rho(0.5f * (cc + right(c0, cx, e)))) * ((right(p0, px, e) - pc) * a.inv_h);
    float gy_s = 0.0f, gy_n = 0.0f;
    if (r.j > 0) gy_s = qdiv(a.rho0, rho(0.5f * (cs.e[e] + cc))) * ((pc - ps.e[e]) * a.inv_h);
    if (r.j < ny - 1) gy_n = qdiv(a.rho0, rho(0.5f * (cc + cn.e[e]))) * ((pn.e[e] - pc) * a.inv_h);
    const float div_g = (gx_e - gx_w) * a.inv_h + (gy_n - gy_s) * a.inv_h;
    const float div_u = (right(us, ux, e) - us.e[e]) * a.inv_h + (vsn.e[e] - vs.e[e]) * a.inv_h;
    rhs.e[e] = (a.rho0 * a.inv_dt) * div_u - div_g;
  }
  if (r.act) {
    st4(d.rhs, r.q, rhs);
    st4(d.phat, r.q, p0);
  }
}

__global__ void IBPF_CELL_BOUNDS kq_correct(const InstDev<float>* __restrict__ I, const int2* __restrict__ blk,
                                            int nblk, int cur) {
  IBPF_QUAD_PROLOGUE
  const float *C = d.C[1 - cur], *dP = d.dp, *phat = d.phat;
  float *uss = d.U[1 - cur], *vss = d.V[1 - cur];
  auto rho = [&](float cc) { return a.rho_a + a.rho_b * clamp1(cc); };
  const V4 c0 = ld4(C, r.q), cs = ld4(C, r.s);
  const V4 ph = ld4(phat, r.q), phs = ld4(phat, r.s);
  const V4 dp = ld4(dP, r.q), dps = ld4(dP, r.s);
  const V4 us = ld4(uss, r.q), vs = ld4(vss, r.q);
  const X2 cx = xnb2(c0, r, d.nx, [&](size_t q) { return C[q]; });
  const X2 phx = xnb2(ph, r, d.nx, [&](size_t q) { return phat[q]; });
  const X2 dpx = xnb2(dp, r, d.nx, [&](size_t q) { return dP[q]; });
  const V4 lo = d.Clo[1 - cur] ? ld4(d.Clo[1 - cur], r.q) : V4{{0.0f, 0.0f, 0.0f, 0.0f}};
  int bad = 0;
  V4 un, vn;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float cc = c0.e[e];
    {
      const float rho_f = rho(0.5f * (left(c0, cx, e) + cc));
      un.e[e] = us.e[e] - a.dt * (qdiv((ph.e[e] - left(ph, phx, e)) * a.inv_h, rho_f) +
                                  a.inv_rho0 * ((dp.e[e] - left(dp, dpx, e)) * a.inv_h));
      bad |= !isfinite(un.e[e]);
    }
    if (r.j >= 1) {
      const float rho_f = rho(0.5f * (cs.e[e] + cc));
      vn.e[e] = vs.e[e] - a.dt * (qdiv((ph.e[e] - phs.e[e]) * a.inv_h, rho_f) +
                                  a.inv_rho0 * ((dp.e[e] - dps.e[e]) * a.inv_h));
      bad |= !isfinite(vn.e[e]);
    }
    bad |= !isfinite(cc);
  }
  float s_hi = 0.0f, s_lo = 0.0f;
  if (r.act) {
    st4(uss, r.q, un);
    if (r.j >= 1) st4(vss, r.q, vn);
    if (bad) atomicOr(d.status, 1);
    s_hi = c0.e[0];
    s_lo = lo.e[0];
#pragma unroll
    for (int e = 1; e < 4; ++e) pair_add(s_hi, s_lo, c0.e[e], lo.e[e]);
  }
  const int ntiles = d.gx * ((d.ny + kTileH - 1) / kTileH);
  tile_mass<float, kTileX * kTileY>(s_hi, s_lo, w_.y, ntiles, d.partial, d.ticket, d.mass);
}
// explicit Cahn-Hilliard variant: kx_phi2 and kx_update on runs of four cells
__device__ __forceinline__ float flux_div_q(const StepArgs<float>& a, const Run2& r, int ny,
                                            const V4& c, const X2& cx, const V4& cn, const V4& cs,
                                            const V4& u, const X2& ux, const V4& v, const V4& vn,
                                            int e) {
  const float c0 = c.e[e];
  const float fx_w = u.e[e] * (0.5f * (left(c, cx, e) + c0));
  const float fx_e = right(u, ux, e) * (0.5f * (c0 + right(c, cx, e)));
  float fy_s = 0.0f, fy_n = 0.0f;
  if (r.j > 0) fy_s = v.e[e] * (0.5f * (cs.e[e] + c0));
  if (r.j < ny - 1) fy_n = vn.e[e] * (0.5f * (c0 + cn.e[e]));
  return (fx_e - fx_w) * a.inv_h + (fy_n - fy_s) * a.inv_h;
}

__global__ void IBPF_CELL_BOUNDS kq_phi2(const InstDev<float>* __restrict__ I, const int2* __restrict__ blk,
                                         int nblk, int cur) {
  IBPF_QUAD_PROLOGUE
  const float *C = d.C[cur], *Co = d.C[1 - cur], *uo = d.U[1 - cur], *vo = d.V[1 - cur];
  const int nx = d.nx;
  const V4 c = ld4(C, r.q), cn = ld4(C, r.n), cs = ld4(C, r.s);
  const V4 o = ld4(Co, r.q), on = ld4(Co, r.n), os = ld4(Co, r.s);
  const V4 u = ld4(uo, r.q), v = ld4(vo, r.q), vn = ld4(vo, r.q + nx);
  const X2 cx = xnb2(c, r, nx, [&](size_t q) { return C[q]; });
  const X2 ox = xnb2(o, r, nx, [&](size_t q) { return Co[q]; });
  const X2 ux = xnb2(u, r, nx, [&](size_t q) { return uo[q]; });
  const V4 pn = map4([&](int e) {
    const float c0 = c.e[e];
    return (c0 * c0 * c0 - c0) - a.eta2 * lap5q(a, c, cx, cn, cs, e);
  });
  const V4 po = map4([&](int e) {
    const float c0 = o.e[e];
    return (c0 * c0 * c0 - c0) - a.eta2 * lap5q(a, o, ox, on, os, e);
  });
  const V4 ao = map4([&](int e) { return -flux_div_q(a, r, d.ny, o, ox, on, os, u, ux, v, vn, e); });
  if (r.act) {
    st4(d.phi, r.q, pn);
    st4(d.rhs, r.q, po);
    st4(d.Q, r.q, ao);
  }
}

__global__ void IBPF_CELL_BOUNDS kq_update(const InstDev<float>* __restrict__ I, const int2* __restrict__ blk,
                                           int nblk, int cur) {
  IBPF_QUAD_PROLOGUE
  const float *C = d.C[cur], *u = d.U[cur], *v = d.V[cur], *ph = d.phi, *po = d.rhs;
  const int nx = d.nx;
  const V4 c = ld4(C, r.q), cn = ld4(C, r.n), cs = ld4(C, r.s);
  const V4 uu = ld4(u, r.q), vv = ld4(v, r.q), vn = ld4(v, r.q + nx);
  const V4 f = ld4(ph, r.q), fn = ld4(ph, r.n), fs = ld4(ph, r.s);
  const V4 g = ld4(po, r.q), gn = ld4(po, r.n), gs = ld4(po, r.s);
  const V4 ao = ld4(d.Q, r.q);
  const V4 lo = d.Clo[cur] ? ld4(d.Clo[cur], r.q) : V4{{0.0f, 0.0f, 0.0f, 0.0f}};
  const X2 cx = xnb2(c, r, nx, [&](size_t q) { return C[q]; });
  const X2 ux = xnb2(uu, r, nx, [&](size_t q) { return u[q]; });
  const X2 fx = xnb2(f, r, nx, [&](size_t q) { return ph[q]; });
  const X2 gx = xnb2(g, r, nx, [&](size_t q) { return po[q]; });
  V4 hi, nlo;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float Fn = -flux_div_q(a, r, d.ny, c, cx, cn, cs, uu, ux, vv, vn, e) +
                     lap5q(a, f, fx, fn, fs, e) * a.inv_pe;
    const float Fo = ao.e[e] + lap5q(a, g, gx, gn, gs, e) * a.inv_pe;
    float h = c.e[e], l = lo.e[e];
    pair_add(h, l, a.dt * (1.5f * Fn - 0.5f * Fo), 0.0f);
    hi.e[e] = h;
    nlo.e[e] = l;
  }
  if (r.act) {
    st4(d.C[1 - cur], r.q, hi);
    if (d.Clo[1 - cur]) st4(d.Clo[1 - cur], r.q, nlo);
  }
}
#undef IBPF_QUAD_PROLOGUE

// ------------------------------------------- a1 + a2, explicit variant (Eq. ExpCH)
// C^{n+1} = C^n + dt (3/2 F^n - 1/2 F^{n-1}),  F = -div(u C_f) + (1/Pe) lap(phi), F^{n-1}
// from the level n-1 fields; phi^n = phi(C^n) and phi^{n-1} = phi(C^{n-1}) with their
// zero-gradient ghost fills.  Three launches:
//   kx_phi2      phi^n -> phi, phi^{n-1} -> rhs, A^{n-1} = -div(u^{n-1} C^{n-1}_f) -> Q
//   kx_fill_phi2 ghost values of phi and rhs (phi_G = phi_M)
//   kx_update    C^{n+1} into the C^{n-1} slot (compensated in FP32); reads C^{n-1} only
//                through Q and rhs, so writing the slot in place is safe
// div(u C_f) with face means of C and no flux through the x2 walls, as in ch_rhs_cell.
template <typename T>
__device__ __forceinline__ T flux_div_cell(const StepArgs<T>& a, const T* __restrict__ C,
                                           const T* __restrict__ u, const T* __restrict__ v,
                                           int i, int j) {
  const int nx = a.nx, ny = a.ny;
  const int im = wrap_m(i, nx), ip = wrap_p(i, nx);
  const size_t r = (size_t)j * nx;
  const T c0 = C[r + i];
  const T fx_w = u[r + i] * (T(0.5) * (C[r + im] + c0));
  const T fx_e = u[r + ip] * (T(0.5) * (c0 + C[r + ip]));
  T fy_s = T(0), fy_n = T(0);
  if (j > 0) fy_s = v[r + i] * (T(0.5) * (C[r - nx + i] + c0));
  if (j < ny - 1) fy_n = v[r + nx + i] * (T(0.5) * (c0 + C[r + nx + i]));
  return (fx_e - fx_w) * a.inv_h + (fy_n - fy_s) * a.inv_h;
}

template <typename T>
__device__ __forceinline__ T lap5_cell(const StepArgs<T>& a, const T* __restrict__ f, int i, int j) {
  const int nx = a.nx, ny = a.ny;
  const size_t r = (size_t)j * nx;
  const int js = j > 0 ? j - 1 : 0, jn = j < ny - 1 ? j + 1 : ny - 1;
  return (((f[r + wrap_p(i, nx)] + f[r + wrap_m(i, nx)]) + (f[(size_t)jn * nx + i] + f[(size_t)js * nx + i])) -
          T(4) * f[r + i]) * a.inv_h2;
}

template <typename T>
__global__ void IBPF_CELL_BOUNDS kx_phi2(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                                         int nblk, int cur) {
  const int b_ = blockIdx.x;
  if (b_ >= nblk) return;
  const int2 w_ = blk[b_];
  const InstDev<T>& d = I[w_.x];
  int i, jb;
  tile_base(d, w_.y, i, jb);
  T o_pn[kRowsPerThread], o_po[kRowsPerThread], o_a[kRowsPerThread];
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
    const int j = jb + q * kTileY;
    if (i < d.nx && j < d.ny) {
      o_pn[q] = chem_pot_cell(d.a, d.C[cur], i, j);
      o_po[q] = chem_pot_cell(d.a, d.C[1 - cur], i, j);
      o_a[q] = -flux_div_cell(d.a, d.C[1 - cur], d.U[1 - cur], d.V[1 - cur], i, j);
    }
  }
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
    const int j = jb + q * kTileY;
    if (i < d.nx && j < d.ny) {
      const size_t c = (size_t)j * d.nx + i;
      d.phi[c] = o_pn[q];
      d.rhs[c] = o_po[q];
      d.Q[c] = o_a[q];
    }
  }
}

template <typename T>
__global__ void kx_fill_phi2(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk, int nblk) {
  const int b_ = blockIdx.x;
  if (b_ >= nblk) return;
  const int2 w_ = blk[b_];
  const InstDev<T>& d = I[w_.x];
  const int g = w_.y * kGhostChunk + threadIdx.x;
  if (g < d.tab.ng) {
    fill_phi_ghost(d.tab, d.phi, g);
    fill_phi_ghost(d.tab, d.rhs, g);
  }
}

template <typename T>
__global__ void IBPF_CELL_BOUNDS kx_update(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                                           int nblk, int cur) {
  const int b_ = blockIdx.x;
  if (b_ >= nblk) return;
  const int2 w_ = blk[b_];
  const InstDev<T>& d = I[w_.x];
  int i, jb;
  tile_base(d, w_.y, i, jb);
  T o_d[kRowsPerThread];
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
    const int j = jb + q * kTileY;
    if (i < d.nx && j < d.ny) {
      const size_t c = (size_t)j * d.nx + i;
      const T Fn = -flux_div_cell(d.a, d.C[cur], d.U[cur], d.V[cur], i, j) +
                   lap5_cell(d.a, d.phi, i, j) * d.a.inv_pe;
      const T Fo = d.Q[c] + lap5_cell(d.a, d.rhs, i, j) * d.a.inv_pe;
      o_d[q] = d.a.dt * (T(1.5) * Fn - T(0.5) * Fo);
    }
  }
#pragma unroll
  for (int q = 0; q < kRowsPerThread; ++q) {
    const int j = jb + q * kTileY;
    if (i < d.nx && j < d.ny) {
      const size_t c = (size_t)j * d.nx + i;
      T hi = d.C[cur][c];
      T lo = d.Clo[cur] ? d.Clo[cur][c] : T(0);
      pair_add(hi, lo, o_d[q], T(0));   // FP64: plain addition
      d.C[1 - cur][c] = hi;
      if (d.Clo[1 - cur]) d.Clo[1 - cur][c] = lo;
    }
  }
}

template <typename T>
int step_batch_t(const Ctx& c, const BatchPlan& plan, int cur, cudaStream_t s, Recorder* rec) {
  const InstDev<T>* I = reinterpret_cast<const InstDev<T>*>(plan.d_inst);
  const dim3 tile(kTileX, kTileY);
  const int nc = plan.nblk[kFamCell], ng = plan.nblk[kFamGhost], nf = plan.nblk[kFamFace];
  const int2* bc = plan.d_blk[kFamCell];
  const int2* bg = plan.d_blk[kFamGhost];
  const int2* bf = plan.d_blk[kFamFace];
  int launches = 0;
  auto mark = [&](const char* n) {
    ++launches;
    if (rec) rec->mark(n, s);
  };
  // a1 + a2: CH right-hand side, then the solve (or the explicit update); C^{n+1} lands in
  // slot 1 - cur
  if (c.ch_scheme == IB_PF_CH_EXPLICIT) {
    if constexpr (sizeof(T) == 4) kq_phi2<<<nc, tile, 0, s>>>(I, bc, nc, cur);
    else kx_phi2<T><<<nc, tile, 0, s>>>(I, bc, nc, cur);
    mark("ch_phi2");
    if (ng > 0) {
      kx_fill_phi2<T><<<ng, kGhostChunk, 0, s>>>(I, bg, ng);
      mark("ch_fill2");
    }
    if constexpr (sizeof(T) == 4) kq_update<<<nc, tile, 0, s>>>(I, bc, nc, cur);
    else kx_update<T><<<nc, tile, 0, s>>>(I, bc, nc, cur);
    mark("ch_explicit");
  } else {
    if constexpr (sizeof(T) == 4) kq_ch_h<<<nc, tile, 0, s>>>(I, bc, nc, cur);
    else kb_ch_h<T><<<nc, tile, 0, s>>>(I, bc, nc, cur);
    mark("ch_h");
    if (ng > 0) {
      kb_ch_wall<T><<<ng, kGhostChunk, 0, s>>>(I, bg, ng, cur);
      mark("ch_wall");
    }
    if constexpr (sizeof(T) == 4) kq_ch_rhs<<<nc, tile, 0, s>>>(I, bc, nc, cur);
    else kb_ch_rhs<T><<<nc, tile, 0, s>>>(I, bc, nc, cur);
    mark("ch_rhs");
    launches += spectral_solve_batch<T>(plan, 0, cur, s, rec);
  }
  // a3: contact-angle ghost fill
  if (ng > 0) {
    kb_fill_C<T><<<ng, kGhostChunk, 0, s>>>(I, bg, ng, cur, 0);
    mark("fill_C");
    if (c.dynamic) {
      kb_fill_C<T><<<ng, kGhostChunk, 0, s>>>(I, bg, ng, cur, 1);
      mark("fill_C");
    }
  }
  // a4: chemical potential and its ghost fill
  if constexpr (sizeof(T) == 4) kq_chem_pot<<<nc, tile, 0, s>>>(I, bc, nc, cur);
  else kb_chem_pot<T><<<nc, tile, 0, s>>>(I, bc, nc, cur);
  mark("chem_pot");
  if (ng > 0) {
    kb_fill_phi<T><<<ng, kGhostChunk, 0, s>>>(I, bg, ng);
    mark("fill_phi");
  }
  // a5: predictor + penalisation, u** into slot 1 - cur (semi-implicit: the right-hand sides,
  // then the two velocity Helmholtz solves, whose inverse row transforms penalise)
  if (c.ns_scheme == IB_PF_NS_SEMI_IMPLICIT) {
    kb_predict<T, true><<<nc, tile, 0, s>>>(I, bc, nc, cur);
    mark("predict");
    launches += spectral_solve_batch<T>(plan, 2, cur, s, rec);
    launches += spectral_solve_batch<T>(plan, 3, cur, s, rec);
  } else {
    kb_predict<T, false><<<nc, tile, 0, s>>>(I, bc, nc, cur);
    mark("predict");
  }
  // a6: velocity ghost fill and face re-interpolation
  if (ng > 0) {
    kb_fill_u<T><<<ng, kGhostChunk, 0, s>>>(I, bg, ng, cur);
    mark("fill_u");
  }
  if (nf > 0) {
    kb_face_values<T><<<nf, kGhostChunk, 0, s>>>(I, bf, nf, cur);
    mark("face_values");
    kb_face_scatter<T><<<nf, kGhostChunk, 0, s>>>(I, bf, nf, cur);
    mark("face_scatter");
  }
  // a7: Poisson right-hand side and solve, P^{n+1} into slot 1 - cur
  if constexpr (sizeof(T) == 4) kq_poisson_rhs<<<nc, tile, 0, s>>>(I, bc, nc, cur);
  else kb_poisson_rhs<T><<<nc, tile, 0, s>>>(I, bc, nc, cur);
  mark("poisson_rhs");
  launches += spectral_solve_batch<T>(plan, 1, cur, s, rec);
  // a8: correction, status, mass
  if constexpr (sizeof(T) == 4) kq_correct<<<nc, tile, 0, s>>>(I, bc, nc, cur);
  else kb_correct<T><<<nc, tile, 0, s>>>(I, bc, nc, cur);
  mark("correct");
  return launches;
}

template <typename T>
cudaError_t batch_setup_t(Ctx& c, BatchPlan& plan) {
  using C2 = typename C2T<T>::type;
  const int n = (int)c.inst.size();
  std::vector<InstDev<T>> host(n);
  std::vector<int2> fam[kNumFam];
  int rmax[2] = {0, 0}, cmax[2] = {0, 0};   // longest row / column per transform class
  int dmax[2] = {0, 0};                     // longest doubled column (DST-I) per class
  plan.max_nx = plan.max_ny = 0;
  for (int k = 0; k < n; ++k) {
    Instance& in = c.inst[k];
    InstDev<T>& d = host[k];
    d.nx = in.nx;
    d.ny = in.ny;
    d.lognx = in.lognx;
    d.logny = in.logny;
    d.gx = (in.nx + kTileX - 1) / kTileX;
    d.a = make_args<T>(in);
    for (int q = 0; q < 2; ++q) {
      d.C[q] = (T*)in.C[q];
      d.Clo[q] = (T*)in.Clo[q];
      d.U[q] = (T*)in.U[q];
      d.V[q] = (T*)in.V[q];
      d.P[q] = (T*)in.P[q];
    }
    d.Hu = (T*)in.Hu;
    d.Hv = (T*)in.Hv;
    d.Q = (T*)in.Q;
    d.phi = (T*)in.phi;
    d.rhs = (T*)in.rhs;
    d.phat = (T*)in.phat;
    d.dp = (T*)in.dp;
    d.spec = (C2*)in.spec;
    d.gu = (T*)in.gu;
    d.gv = (T*)in.gv;
    d.fval = (T*)in.fval;
    d.ci = (double*)in.ci;
    d.gq = (T*)in.gq;
    d.tab = in.tab;
    d.lamx = in.lamx;
    d.lamy = in.lamy;
    d.lamx_f = in.lamx_f;
    d.lamy_f = in.lamy_f;
    d.twx = (const C2*)in.twx;
    d.twy = (const C2*)in.twy;
    d.wd = (const C2*)in.wdct;
    d.s_eta2 = in.prm.S / (in.prm.Cn * in.prm.Cn);
    // semi-implicit predictor: a = dt nu0 / 2, nu0 = (mu_l/rho_l + mu_g/rho_g) / (2 Re)
    d.a_visc = 0.5 * in.prm.dt * 0.5 * (1.0 + (1.0 / in.prm.mu_ratio) / (1.0 / in.prm.rho_ratio)) / in.prm.Re;
    d.lam_s2 = in.lam_s2;
    d.lam_d1 = in.lam_d1;
    d.lam_s2_f = in.lam_s2_f;
    d.lam_d1_f = in.lam_d1_f;
    d.tw2 = (const C2*)in.tw2;
    d.c0 = 1.5 * in.prm.Pe / (in.prm.Cn * in.prm.Cn * in.prm.dt);
    d.partial = in.partial;
    d.ticket = in.ticket;
    d.mass = in.mass;
    d.status = in.status;
    const int ntiles = d.gx * ((in.ny + kTileH - 1) / kTileH);
    for (int b = 0; b < ntiles; ++b) fam[kFamCell].push_back(make_int2(k, b));
    const int rp = fft_per_block(in.nx), cp = fft_per_block(in.ny);
    const int rl = fft_threads(in.nx) == kFftLargeThreads, cl = fft_threads(in.ny) == kFftLargeThreads;
    for (int b = 0; b < (in.ny / 2 + rp - 1) / rp; ++b)
      fam[rl ? kFamRowsL : kFamRows].push_back(make_int2(k, b));
    rmax[rl] = in.nx > rmax[rl] ? in.nx : rmax[rl];
    const int ncg = (in.nx / 2 + 1 + cp - 1) / cp;
    for (int b = 0; b < ncg; ++b) fam[cl ? kFamColsL : kFamCols].push_back(make_int2(k, b));
    cmax[cl] = in.ny > cmax[cl] ? in.ny : cmax[cl];
    if (c.ns_scheme == IB_PF_NS_SEMI_IMPLICIT) {
      // DST-I columns: complex FFTs of 2 ny points
      const int dp = fft_per_block(2 * in.ny), dl = fft_threads(2 * in.ny) == kFftLargeThreads;
      for (int b = 0; b < (in.nx / 2 + 1 + dp - 1) / dp; ++b)
        fam[dl ? kFamD1L : kFamD1].push_back(make_int2(k, b));
      dmax[dl] = 2 * in.ny > dmax[dl] ? 2 * in.ny : dmax[dl];
    }
    for (int b = 0; b < (in.tab.ng + kGhostChunk - 1) / kGhostChunk; ++b)
      fam[kFamGhost].push_back(make_int2(k, b));
    const int nf = in.tab.nfu + in.tab.nfv;
    for (int b = 0; b < (nf + kGhostChunk - 1) / kGhostChunk; ++b)
      fam[kFamFace].push_back(make_int2(k, b));
    plan.max_nx = in.nx > plan.max_nx ? in.nx : plan.max_nx;
    plan.max_ny = in.ny > plan.max_ny ? in.ny : plan.max_ny;
  }
  cudaError_t e;
  if constexpr (sizeof(T) == 8) {
    for (int k = 0; k < n; ++k) {
      host[k].au = c.inst[k].tab.alpha_u;
      host[k].av = c.inst[k].tab.alpha_v;
    }
  } else {
    // the FP32 form reads the face fractions in FP32 (rounded once from the FP64 tables)
    size_t tot = 0;
    for (int k = 0; k < n; ++k) tot += (size_t)(2 * c.inst[k].ny + 1) * c.inst[k].nx;
    e = cudaMalloc(&plan.alpha_f, sizeof(float) * tot);
    if (e != cudaSuccess) return e;
    float* dst = (float*)plan.alpha_f;
    std::vector<double> hd;
    std::vector<float> hf;
    for (int k = 0; k < n; ++k) {
      const Instance& in = c.inst[k];
      const size_t nu = (size_t)in.ny * in.nx, nv = nu + in.nx;
      hd.resize(nu + nv);
      e = cudaMemcpy(hd.data(), in.tab.alpha_u, sizeof(double) * nu, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return e;
      e = cudaMemcpy(hd.data() + nu, in.tab.alpha_v, sizeof(double) * nv, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return e;
      hf.assign(hd.begin(), hd.end());
      e = cudaMemcpy(dst, hf.data(), sizeof(float) * (nu + nv), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return e;
      host[k].au = (const T*)dst;
      host[k].av = (const T*)(dst + nu);
      dst += nu + nv;
    }
  }
  e = cudaMalloc(&plan.d_inst, sizeof(InstDev<T>) * n);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(plan.d_inst, host.data(), sizeof(InstDev<T>) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  for (int f = 0; f < kNumFam; ++f) {
    plan.nblk[f] = (int)fam[f].size();
    e = cudaMalloc((void**)&plan.d_blk[f], sizeof(int2) * (fam[f].empty() ? 1 : fam[f].size()));
    if (e != cudaSuccess) return e;
    if (!fam[f].empty()) {
      e = cudaMemcpy(plan.d_blk[f], fam[f].data(), sizeof(int2) * fam[f].size(),
                     cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return e;
    }
  }
  for (int c = 0; c < 2; ++c) {
    const int eb = 8 * (c ? kFftLargeThreads : kFftSmallThreads);
    plan.rows_smem[c] = sizeof(C2) * (fft_buf(eb) + rmax[c] / 2);
    plan.cols_smem[c] = cols_smem_bytes<T>(cmax[c], eb, 8);
    // DST-I blocks: points, twiddles of the doubled length, one eigenvalue part per column
    plan.d1_smem[c] = sizeof(C2) * (size_t)(fft_buf(eb) + dmax[c] / 2) + sizeof(T) * (size_t)(eb / 16);
  }
  return cudaSuccess;
}

template <typename T>
int mass_t(Instance& in, const void* C, const void* Clo, cudaStream_t s) {
  const int n = in.nx * in.ny * in.nz;
  int nb = (n + 255) / 256;
  if (nb > in.nblk_red) nb = in.nblk_red;
  k_mass<T><<<nb, 256, 0, s>>>(n, (const T*)C, (const T*)Clo, in.partial, in.ticket, in.mass);
  return 1;
}

}  // namespace

cudaError_t batch_setup(Ctx& c, BatchPlan& plan) {
  return c.precision == IB_PF_FP64 ? batch_setup_t<double>(c, plan) : batch_setup_t<float>(c, plan);
}

void batch_free(BatchPlan& plan) {
  if (plan.d_inst) cudaFree(plan.d_inst);
  if (plan.alpha_f) cudaFree(plan.alpha_f);
  for (int f = 0; f < kNumFam; ++f)
    if (plan.d_blk[f]) cudaFree(plan.d_blk[f]);
  plan = BatchPlan();
}

int step_batch(const Ctx& c, const BatchPlan& plan, int cur, cudaStream_t s, Recorder* rec) {
  return c.precision == IB_PF_FP64 ? step_batch_t<double>(c, plan, cur, s, rec)
                                   : step_batch_t<float>(c, plan, cur, s, rec);
}

int mass_reduce(Instance& in, int precision, const void* C, const void* Clo, cudaStream_t s) {
  return precision == IB_PF_FP64 ? mass_t<double>(in, C, Clo, s) : mass_t<float>(in, C, Clo, s);
}

}  // namespace ibpf
