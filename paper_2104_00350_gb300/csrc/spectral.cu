// Separable spectral solves of the hybrid IB / phase-field step (Appendix A.1 and
// Eq. PressurePoisson): the 5-point Laplacian with periodic x1 and zero-gradient x2 walls
// is diagonal in the basis  exp(2 pi i k x1 / Lx)  x  cos(pi m (j + 1/2) / ny).
//
// A solve is three kernels:
//   rows_fwd : real FFT of every x1 row (two rows packed into one complex FFT),
//   cols     : per spectral column k, cosine transform (DCT-II) along x2, division by the
//              symbol, inverse cosine transform (the last forward axis and the first
//              inverse axis fused in shared memory),
//   rows_inv : inverse real FFT of every row (two rows per complex FFT).
// FFTs are Stockham autosort transforms, radix 8 in registers with one radix-4 or radix-2
// pass for the remaining factor, exchanging through shared memory between passes.
// The cosine transforms use an N-point complex FFT with the even/odd reordering
// v_n = x_{2n}, v_{N-1-n} = x_{2n+1} (Makhoul's algorithm).
#include <cmath>
#include <vector>

#include "batch.h"
#include "ibpf_internal.h"

namespace ibpf {
namespace {

template <typename C2>
__device__ __forceinline__ C2 cmul(C2 a, C2 b) {
  C2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C2>
__device__ __forceinline__ C2 cadd(C2 a, C2 b) { C2 r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C2>
__device__ __forceinline__ C2 csub(C2 a, C2 b) { C2 r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C2>
__device__ __forceinline__ C2 cconj(C2 a) { a.y = -a.y; return a; }

// ------------------------------------------------------------------ Stockham FFT
// cnt independent FFTs of length N = 2^LOGN, stored back to back in the shared buffer x at
// padded slots pad(i) (one pad slot per 16 points, so that the strided stores of the early
// passes and the unit-stride loads of the next pass both spread over the 32 banks).
// Input and output are in natural order (Stockham autosort).  Each pass of radix R takes
// groups j < N/R: v_r = x[j + r N/R] times the twiddle W_{Ns R}^{r (j mod Ns)}, an R-point
// DFT in registers, stored at ((j - j mod Ns) R + j mod Ns) + r Ns, where Ns is the product
// of the radices of the earlier passes (radix 8, then one radix-4 or radix-2 pass).
// A pass loads all its groups into registers, synchronises, stores, synchronises.
// Forward: W = exp(-2 pi i/N); INV: conjugate twiddles, no 1/N.  tw[m] = exp(-2 pi i m/N),
// m < N/2, the other half by W^{m + N/2} = -W^m.
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }

// Slot of point i of transform f.  P = 8 (8 points per thread): transforms back to back,
// pad(f N + i).  P > 8 (more points per thread): transform f starts at f (N + N/16 + 1),
// one slot more than its padded length, so that a phase in which consecutive threads take
// the same point of consecutive transforms hits distinct banks.
template <int N, int P>
__device__ __forceinline__ int xslot(int f, int i) {
  if constexpr (P > 8) return f * (N + (N >> 4) + 1) + pad(i);
  else return pad(f * N + i);
}
// complex slots of a block's transform buffer for e points of length-n transforms
__host__ __device__ constexpr int xbuf(int e, int n, int p) {
  return p > 8 ? (e / n) * (n + (n >> 4) + 1) : fft_buf(e);
}

template <bool INV, typename C2>
__device__ __forceinline__ C2 mul_mi(C2 a) {   // a times -i (forward) or +i (inverse)
  C2 r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

template <int R, bool INV, typename T, typename C2>
__device__ __forceinline__ void dft_reg(C2* v) {
  if constexpr (R == 2) {
    const C2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const C2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const C2 s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  } else {
    static_assert(R == 8, "radix 2, 4 or 8");
    C2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft_reg<4, INV, T>(e);
    dft_reg<4, INV, T>(o);
    const T c = T(0.70710678118654752440);   // cos(pi/4)
    C2 w1, w3;                                 // W8^1 o_1 and W8^3 o_3
    if (INV) {
      w1.x = c * (o[1].x - o[1].y); w1.y = c * (o[1].x + o[1].y);
      w3.x = -c * (o[3].x + o[3].y); w3.y = c * (o[3].x - o[3].y);
    } else {
      w1.x = c * (o[1].x + o[1].y); w1.y = c * (o[1].y - o[1].x);
      w3.x = c * (o[3].y - o[3].x); w3.y = -c * (o[3].x + o[3].y);
    }
    const C2 w2 = mul_mi<INV>(o[2]);
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);   v[5] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);   v[6] = csub(e[2], w2);
    v[3] = cadd(e[3], w3);   v[7] = csub(e[3], w3);
  }
}

template <int LOGN, int R, int NS, bool INV, int THREADS, typename T, int P, typename C2>
__device__ __forceinline__ void stockham_pass(C2* x, const C2* __restrict__ tw, int cnt) {
  constexpr int N = 1 << LOGN, NR = N / R, HALF = N / 2;
  static_assert(N <= P * THREADS, "a block holds P points per thread");
  constexpr int Q = P / R;                    // groups per thread
  constexpr int TSTEP = N / (NS * R);         // twiddle index step
  const int ng = cnt * NR;
  C2 v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int g = threadIdx.x + q * THREADS;
    if (g < ng) {
      const int f = g / NR, j = g % NR;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = x[xslot<N, P>(f, j + r * NR)];
      if constexpr (NS > 1) {
        const int k = j % NS;
        auto tw_at = [&](int m) {   // W^m, m < N
          C2 w = tw[m & (HALF - 1)];
          if (m >= HALF) { w.x = -w.x; w.y = -w.y; }
          if (INV) w.y = -w.y;
          return w;
        };
        if constexpr (R == 8) {
          // W^k, W^2k, W^4k from the table, the other four by products (at most two
          // roundings deep): a third of the table reads of a radix-8 butterfly
          const C2 w1 = tw_at(k * TSTEP), w2 = tw_at(2 * k * TSTEP), w4 = tw_at(4 * k * TSTEP);
          const C2 w3 = cmul(w1, w2);
          v[q][1] = cmul(v[q][1], w1);
          v[q][2] = cmul(v[q][2], w2);
          v[q][3] = cmul(v[q][3], w3);
          v[q][4] = cmul(v[q][4], w4);
          v[q][5] = cmul(v[q][5], cmul(w1, w4));
          v[q][6] = cmul(v[q][6], cmul(w2, w4));
          v[q][7] = cmul(v[q][7], cmul(w3, w4));
        } else {
#pragma unroll
          for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], tw_at(r * k * TSTEP));
        }
      }
      dft_reg<R, INV, T>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int g = threadIdx.x + q * THREADS;
    if (g < ng) {
      const int f = g / NR, j = g % NR, k = j % NS;
      const int d = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) x[xslot<N, P>(f, d + r * NS)] = v[q][r];
    }
  }
  __syncthreads();
}

// P: points per thread (8 by default)
template <int LOGN, int DONE, bool INV, int THREADS, typename T, int P = 8, typename C2>
__device__ __forceinline__ void stockham(C2* x, const C2* __restrict__ tw, int cnt) {
  if constexpr (DONE < LOGN) {
    constexpr int LR = (LOGN - DONE) >= 3 ? 3 : (LOGN - DONE);
    stockham_pass<LOGN, (1 << LR), (1 << DONE), INV, THREADS, T, P>(x, tw, cnt);
    stockham<LOGN, DONE + LR, INV, THREADS, T, P>(x, tw, cnt);
  }
}

// Forward real FFT of the cnt row pairs (ra + 2f, ra + 2f + 1), f < cnt, of in (ny x nx)
// into spec (ny rows of sp >= nx/2+1 points).  Per pair z = row_a + i row_b;
// A_k = (Z_k + conj Z_{N-k})/2,  B_k = (Z_k - conj Z_{N-k})/(2i).
template <typename T, int LOGN, int THREADS>
__device__ void rows_fwd_core(const T* __restrict__ in, typename C2T<T>::type* __restrict__ spec,
                              const typename C2T<T>::type* __restrict__ tw, size_t ra, int cnt,
                              int sp, typename C2T<T>::type* x) {
  using C2 = typename C2T<T>::type;
  constexpr int nx = 1 << LOGN, nh = nx >> 1;
  constexpr int EB = 8 * THREADS;
  C2* tws = x + fft_buf(EB);   // twiddles staged after the data
  for (int t = threadIdx.x; t < nh; t += THREADS) tws[t] = tw[t];
  for (int t = threadIdx.x; t < cnt * nx; t += THREADS) {
    const int f = t >> LOGN, n = t & (nx - 1);
    const size_t r = ra + 2 * f;
    C2 z;
    z.x = in[r * nx + n];
    z.y = in[(r + 1) * nx + n];
    x[pad(t)] = z;
  }
  __syncthreads();
  stockham<LOGN, 0, false, THREADS, T>(x, tws, cnt);
  for (int t = threadIdx.x; t < cnt * (nh + 1); t += THREADS) {
    const int f = t / (nh + 1), k = t - f * (nh + 1);
    const size_t r = ra + 2 * f;
    C2 z = x[pad(f * nx + (k & (nx - 1)))], zc = x[pad(f * nx + ((nx - k) & (nx - 1)))];
    C2 A, B;
    A.x = T(0.5) * (z.x + zc.x);
    A.y = T(0.5) * (z.y - zc.y);
    B.x = T(0.5) * (z.y + zc.y);
    B.y = T(-0.5) * (z.x - zc.x);
    spec[r * sp + k] = A;
    spec[(r + 1) * sp + k] = B;
  }
  __syncthreads();   // the shared buffer may be reused by the caller
}

// (hi, lo) + inc -> (out_hi, out_lo): TwoSum of hi and inc (Knuth), the rounding error
// added to lo, then a FastTwoSum renormalisation.  Only additions, so no contraction.
template <typename T>
__device__ __forceinline__ void two_sum_into(T hi, T inc, T lo, T& out_hi, T& out_lo) {
  const T s = hi + inc;
  const T bb = s - hi;
  const T err = (hi - (s - bb)) + (inc - bb);
  const T l = lo + err;
  const T h2 = s + l;
  out_hi = h2;
  out_lo = l - (h2 - s);
}

// Inverse of rows_fwd_core: Z_k = A_k + i B_k with Hermitian extension (imaginary parts of
// the k = 0 and k = nx/2 bins dropped), z = IFFT(Z)/nx, row_a = Re z, row_b = Im z.
// Epilogue (the solves return increments):
//   kind 0: out = z
//   kind 1: out = a + ((a - b)/3 + z)    (BDF2 predictor (2a - b/2)/1.5 of C plus the
//                                          increment, small terms first; out may alias b)
//   kind 2: delta = z, out = z + a         (pressure increment on top of a = P^)
template <typename T, int LOGN, int THREADS>
__device__ void rows_inv_core(const typename C2T<T>::type* __restrict__ spec, T* out,
                              const typename C2T<T>::type* __restrict__ tw, const EpiArgs& epi,
                              size_t ra, int cnt, int sp, typename C2T<T>::type* x) {
  using C2 = typename C2T<T>::type;
  constexpr int nx = 1 << LOGN, nh = nx >> 1;
  constexpr int EB = 8 * THREADS;
  for (int t = threadIdx.x; t < cnt * nx; t += THREADS) {
    const int f = t >> LOGN, k = t & (nx - 1);
    const size_t r = ra + 2 * f;
    int kk = k <= nh ? k : nx - k;
    C2 A = spec[r * sp + kk], B = spec[(r + 1) * sp + kk];
    if (kk == 0 || kk == nh) {
      A.y = T(0);
      B.y = T(0);
    }
    if (k > nh) {
      A = cconj(A);
      B = cconj(B);
    }
    C2 z;
    z.x = A.x - B.y;
    z.y = A.y + B.x;
    x[pad(t)] = z;
  }
  C2* tws = x + fft_buf(EB);   // twiddles staged after the data
  for (int t = threadIdx.x; t < nh; t += THREADS) tws[t] = tw[t];
  __syncthreads();
  stockham<LOGN, 0, true, THREADS, T>(x, tws, cnt);
  const T inv = T(1) / T(nx);
  const T* ea = reinterpret_cast<const T*>(epi.a);
  const T* eb = reinterpret_cast<const T*>(epi.b);
  T* ed = reinterpret_cast<T*>(epi.delta);
  for (int t = threadIdx.x; t < cnt * nx; t += THREADS) {
    const int f = t >> LOGN, n = t & (nx - 1);
    const size_t r = ra + 2 * f;
    C2 z = x[pad(t)];
    const size_t ia = r * nx + n, ib = (r + 1) * nx + n;
    T va = z.x * inv, vb = z.y * inv;
    if (epi.kind == 1 && epi.out_lo != nullptr) {
      // compensated state: value = hi + lo; new pair by TwoSum, then renormalised
      const T* al = reinterpret_cast<const T*>(epi.a_lo);
      const T* bl = reinterpret_cast<const T*>(epi.b_lo);
      T* ol = reinterpret_cast<T*>(epi.out_lo);
      const T third = T(1.0 / 3.0);
      T lo_a = al[ia], lo_b = al[ib];
      T inc_a = ((ea[ia] - eb[ia]) + (lo_a - bl[ia])) * third + va;
      T inc_b = ((ea[ib] - eb[ib]) + (lo_b - bl[ib])) * third + vb;
      two_sum_into(ea[ia], inc_a, lo_a, va, ol[ia]);
      two_sum_into(ea[ib], inc_b, lo_b, vb, ol[ib]);
    } else if (epi.kind == 1) {
      const T third = T(1.0 / 3.0);
      va = ea[ia] + ((ea[ia] - eb[ia]) * third + va);
      vb = ea[ib] + ((ea[ib] - eb[ib]) * third + vb);
    } else if (epi.kind == 2) {
      ed[ia] = va;
      ed[ib] = vb;
      va = va + ea[ia];
      vb = vb + ea[ib];
    } else if (epi.kind == 3) {
      const T* al = reinterpret_cast<const T*>(epi.alpha);
      va = al[ia] * (ea[ia] + va);
      vb = al[ib] * (ea[ib] + vb);
    }
    out[ia] = va;
    out[ib] = vb;
  }
  __syncthreads();
}

struct SymbolArgs {
  int mode;          // 0: Cahn-Hilliard quartic, 1: Poisson, 2: Helmholtz 1 - c0 L
  double s_eta2;     // S / Cn^2
  double c0;         // 1.5 Pe / (Cn^2 dt)
  const double* lamx;
  const double* lamy;
  const float* lamx_f;   // FP32 path: eigenvalues computed in FP64, rounded once
  const float* lamy_f;
  // 3D: the columns are (y mode, x mode) pairs c = ky * ncx + kx, lamy / lamy_f hold the z
  // eigenvalues (the transformed axis) and lamyp / lamyp_f the periodic y ones; 0 in 2D
  int ncx = 0;
  const double* lamyp = nullptr;
  const float* lamyp_f = nullptr;
  float s_eta2_f = 0.f, c0_f = 0.f;   // FP32 path: s_eta2 and c0 rounded once
};

// Divide X_m by the symbol at eigenvalue L = lm + lc (2D: lm = lamy[m], lc = lamx[k]; 3D:
// (lamz[m] + lamy[ky]) + lamx[kx], summed in that order by the caller).  FP64 path: in FP64.
// FP32 path: in FP32 -- the three terms of L^2 - (S/Cn^2) L + c0 (L <= 0) and the two of L
// are all of one sign, so the FP32 evaluation has no cancellation and keeps FP32 relative
// accuracy (FP64 here would occupy GB300's narrow FP64 pipe for most of the kernel).
template <typename T, typename C2>
__device__ __forceinline__ C2 divide_symbol(C2 X, T L, const SymbolArgs& sym) {
  if constexpr (sizeof(T) == 8) {
    // one correctly rounded reciprocal per point (__drcp_rn / __frcp_rn, the value of 1/x):
    // the quotient is within 1.5 ulp of X / sigma
    double r;
    if (sym.mode == 0) r = __drcp_rn(L * L - sym.s_eta2 * L + sym.c0);
    else if (sym.mode == 2) r = __drcp_rn(1.0 - sym.c0 * L);     // (1 - a L), a = c0
    else r = (L == 0.0) ? 0.0 : __drcp_rn(L);
    X.x = X.x * r;
    X.y = X.y * r;
  } else {
    float r;
    if (sym.mode == 0) r = __frcp_rn(L * L - sym.s_eta2_f * L + sym.c0_f);
    else if (sym.mode == 2) r = __frcp_rn(1.0f - sym.c0_f * L);
    else r = (L == 0.0f) ? 0.0f : __frcp_rn(L);
    X.x = X.x * r;
    X.y = X.y * r;
  }
  return X;
}

// x2 cosine transform, symbol division and inverse cosine transform of the KC =
// fft_per_block(N) spectral columns k0 .. k0 + KC - 1 (columns at or beyond nh1 are zero and
// not stored).  The data are complex; the transform is real so it acts on Re and Im alike.
//   forward  X_m = sum_j x_j cos(pi m (2j+1)/(2N)) via V = FFT(v), v the even/odd reorder:
//            X_m = Re(w_m Vr_m) + i Re(w_m Vi_m), w_m = exp(-i pi m/(2N)),
//            Vr_m = (V_m + conj V_{N-m})/2, Vi_m = (V_m - conj V_{N-m})/(2i);
//   divide   X_m /= sigma(k, m);
//   inverse  Z_m = conj(w_m) (X_m - i X_{N-m}) (X_N = 0), z = IFFT(Z)/N,
//            x_{2n} = z_n, x_{2n+1} = z_{N-1-n}.
// Dynamic shared memory: cols_smem_bytes<T>(N, EB) (points, twiddles, cosine weights and the
// per-column eigenvalue parts).
// FLIP: the sine transform DST-II (velocity components with no-slip ghost rows) by the same
// pipeline: DST-II(x)_{N-k} = DCT-II((-1)^j x_j)_k, so the column is multiplied by (-1)^j on
// load and on store and the eigenvalue table is given in the cosine order k.
template <typename T, int LOGN, int THREADS, int P = 8, bool FLIP = false>
__device__ void cols_core(typename C2T<T>::type* __restrict__ spec, int nh1,
                          const typename C2T<T>::type* __restrict__ tw,
                          const typename C2T<T>::type* __restrict__ wd, const SymbolArgs& sym,
                          int k0, typename C2T<T>::type* xs) {
  using C2 = typename C2T<T>::type;
  constexpr int N = 1 << LOGN, half = N >> 1;
  constexpr int EB = P * THREADS, KC = EB / N;
  static_assert(KC >= 1, "a block holds P points per thread");
  C2* tws = xs + xbuf(EB, N, P);   // FFT twiddles, staged once per block
  C2* wds = tws + half;            // cosine-transform weights
  // per column c: lcs[c] = lamx[kx], lcs[KC + c] = lamy[ky] (3D: columns k = ky ncx + kx;
  // 2D: kx = k, no y part), computed once per block; lms[m]: the transformed axis
  T* lcs = reinterpret_cast<T*>(wds + N);
  const T* lms = sizeof(T) == 8 ? (const T*)sym.lamy : (const T*)sym.lamy_f;
  const T* lam_x = sizeof(T) == 8 ? (const T*)sym.lamx : (const T*)sym.lamx_f;
  const T* lam_y = sizeof(T) == 8 ? (const T*)sym.lamyp : (const T*)sym.lamyp_f;
  for (int t = threadIdx.x; t < half; t += THREADS) tws[t] = tw[t];
  for (int t = threadIdx.x; t < N; t += THREADS) wds[t] = wd[t];
  for (int c = threadIdx.x; c < KC; c += THREADS) {
    const int k = min(k0 + c, nh1 - 1);
    lcs[c] = sym.ncx ? lam_x[k % sym.ncx] : lam_x[k];
    lcs[KC + c] = sym.ncx ? lam_y[k / sym.ncx] : T(0);
  }
  // load: consecutive threads take consecutive columns of one row (KC columns: rows of KC
  // contiguous points); the loads of a chunk of up to 16 points per thread are all issued
  // before their shared-memory stores
  constexpr int LC = P < 16 ? P : 16;
#pragma unroll
  for (int q0 = 0; q0 < P; q0 += LC) {
    C2 ld[LC];
#pragma unroll
    for (int q = 0; q < LC; ++q) {
      const int idx = threadIdx.x + (q0 + q) * THREADS;
      const int cc = idx % KC, r = idx / KC;
      const int k = k0 + cc;
      ld[q].x = T(0);
      ld[q].y = T(0);
      if (k < nh1) ld[q] = spec[(size_t)r * nh1 + k];
      if (FLIP && (r & 1)) {
        ld[q].x = -ld[q].x;
        ld[q].y = -ld[q].y;
      }
    }
#pragma unroll
    for (int q = 0; q < LC; ++q) {
      const int idx = threadIdx.x + (q0 + q) * THREADS;
      const int cc = idx % KC, r = idx / KC;
      const int pos = (r & 1) ? (N - 1 - (r >> 1)) : (r >> 1);
      xs[xslot<N, P>(cc, pos)] = ld[q];
    }
  }
  // L at (column c, mode m), in the order (lamz[m] + lamy[ky]) + lamx[kx] (3D) or
  // lamy[m] + lamx[k] (2D)
  auto eig = [&](int c, int m) -> T {
    return sym.ncx ? (lms[m] + lcs[KC + c]) + lcs[c] : lms[m] + lcs[c];
  };
  __syncthreads();
  stockham<LOGN, 0, false, THREADS, T, P>(xs, tws, KC);
  // pair tasks (m, N - m), m = 0..N/2, of every column
  for (int t = threadIdx.x; t < KC * (half + 1); t += THREADS) {
    const int c = t / (half + 1), m = t - c * (half + 1);
    const int mm = (N - m) & (N - 1);
    const int im = xslot<N, P>(c, m), imm = xslot<N, P>(c, mm);
    const C2 Vm = xs[im], Vmm = xs[imm];
    C2 Xm, Xmm;
    {
      C2 vr, vi, w = wds[m];
      vr.x = T(0.5) * (Vm.x + Vmm.x);
      vr.y = T(0.5) * (Vm.y - Vmm.y);
      vi.x = T(0.5) * (Vm.y + Vmm.y);
      vi.y = T(-0.5) * (Vm.x - Vmm.x);
      Xm.x = w.x * vr.x - w.y * vr.y;
      Xm.y = w.x * vi.x - w.y * vi.y;
    }
    {
      C2 vr, vi, w = wds[mm];
      vr.x = T(0.5) * (Vmm.x + Vm.x);
      vr.y = T(0.5) * (Vmm.y - Vm.y);
      vi.x = T(0.5) * (Vmm.y + Vm.y);
      vi.y = T(-0.5) * (Vmm.x - Vm.x);
      Xmm.x = w.x * vr.x - w.y * vr.y;
      Xmm.y = w.x * vi.x - w.y * vi.y;
    }
    Xm = divide_symbol<T>(Xm, eig(c, m), sym);
    Xmm = divide_symbol<T>(Xmm, eig(c, mm), sym);
    // inverse pre-processing: Z_m = conj(w_m) (X_m - i X_{N-m})
    C2 Zm, Zmm;
    {
      C2 y;   // X_m - i X_{N-m}; X_N = 0 for m = 0
      C2 xo = (m == 0) ? C2{T(0), T(0)} : Xmm;
      y.x = Xm.x + xo.y;
      y.y = Xm.y - xo.x;
      Zm = cmul(cconj(wds[m]), y);
    }
    {
      C2 y;
      C2 xo = (mm == 0) ? C2{T(0), T(0)} : Xm;
      y.x = Xmm.x + xo.y;
      y.y = Xmm.y - xo.x;
      Zmm = cmul(cconj(wds[mm]), y);
    }
    xs[im] = Zm;
    if (mm != m) xs[imm] = Zmm;
  }
  __syncthreads();
  stockham<LOGN, 0, true, THREADS, T, P>(xs, tws, KC);
  const T inv = T(1) / T(N);
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int idx = threadIdx.x + q * THREADS;
    const int cc = idx % KC, r = idx / KC;
    const int kk = k0 + cc;
    const int n = (r & 1) ? (N - 1 - (r >> 1)) : (r >> 1);
    C2 z = xs[xslot<N, P>(cc, n)];
    const T sc = (FLIP && (r & 1)) ? -inv : inv;
    z.x *= sc;
    z.y *= sc;
    if (kk < nh1) spec[(size_t)r * nh1 + kk] = z;
  }
  __syncthreads();
}

// Sine transform DST-I of the interior rows 1 .. N-1 of the KC = 8 THREADS / (2N) spectral
// columns k0 .. (velocity components that vanish on the wall rows), divided by the symbol
// and transformed back: each column is extended oddly to length 2N (e_0 = e_N = 0,
// e_{2N-j} = -e_j), transformed by a complex FFT of length 2N, divided mode by mode by the
// symbol at the folded index min(m, 2N - m) (lam_d1, N + 1 entries; the m = 0 and m = N
// modes vanish), transformed back and scaled by 1/(2N); row 0 is stored as zero.
template <typename T, int LOGN2, int THREADS>
__device__ void dst1_core(typename C2T<T>::type* __restrict__ spec, int nh1,
                          const typename C2T<T>::type* __restrict__ tw2, const SymbolArgs& sym,
                          const T* __restrict__ lam_d1, int k0, typename C2T<T>::type* xs) {
  using C2 = typename C2T<T>::type;
  constexpr int M = 1 << LOGN2, N = M >> 1;
  constexpr int EB = 8 * THREADS, KC = EB / M;
  static_assert(KC >= 1, "a block holds 8 points per thread");
  C2* tws = xs + fft_buf(EB);
  T* lcs = reinterpret_cast<T*>(tws + N);   // lamx of each column
  const T* lam_x = sizeof(T) == 8 ? (const T*)sym.lamx : (const T*)sym.lamx_f;
  for (int t = threadIdx.x; t < N; t += THREADS) tws[t] = tw2[t];
  for (int c = threadIdx.x; c < KC; c += THREADS) lcs[c] = lam_x[min(k0 + c, nh1 - 1)];
  // consecutive threads take consecutive columns of one row
  for (int idx = threadIdx.x; idx < KC * N; idx += THREADS) {
    const int cc = idx % KC, j = idx / KC;
    const int k = k0 + cc;
    C2 v;
    v.x = T(0);
    v.y = T(0);
    if (j > 0 && k < nh1) v = spec[(size_t)j * nh1 + k];
    xs[pad(cc * M + j)] = v;
    C2 w;
    w.x = -v.x;
    w.y = -v.y;
    if (j == 0) w = v;   // e_N = 0 (v is zero here)
    xs[pad(cc * M + (j == 0 ? N : M - j))] = w;
  }
  __syncthreads();
  stockham<LOGN2, 0, false, THREADS, T>(xs, tws, KC);
  for (int t = threadIdx.x; t < KC * M; t += THREADS) {
    const int c = t / M, m = t - c * M;
    const int mm = m <= N ? m : M - m;
    C2 X = xs[pad(c * M + m)];
    if (mm == 0 || mm == N) {
      X.x = T(0);
      X.y = T(0);
    } else {
      X = divide_symbol<T>(X, lam_d1[mm] + lcs[c], sym);
    }
    xs[pad(c * M + m)] = X;
  }
  __syncthreads();
  stockham<LOGN2, 0, true, THREADS, T>(xs, tws, KC);
  const T inv = T(1) / T(M);
  for (int idx = threadIdx.x; idx < KC * N; idx += THREADS) {
    const int cc = idx % KC, j = idx / KC;
    const int k = k0 + cc;
    C2 z = xs[pad(cc * M + j)];
    z.x *= inv;
    z.y *= inv;
    if (j == 0) {
      z.x = T(0);
      z.y = T(0);
    }
    if (k < nh1) spec[(size_t)j * nh1 + k] = z;
  }
  __syncthreads();
}

// Transform lengths select compile-time instantiations: 8 .. 1024 points in 128-thread
// blocks, 2048 and 4096 points in 512-thread blocks.
#define IBPF_CASES_128 IBPF_CASE(3) IBPF_CASE(4) IBPF_CASE(5) IBPF_CASE(6) IBPF_CASE(7) \
  IBPF_CASE(8) IBPF_CASE(9) IBPF_CASE(10)
#define IBPF_CASES_512 IBPF_CASE(11) IBPF_CASE(12)
#define IBPF_DISPATCH(THREADS, LOGN_EXPR)                              \
  if constexpr (THREADS == kFftSmallThreads) {                         \
    switch (LOGN_EXPR) { IBPF_CASES_128 default: break; }              \
  } else {                                                             \
    switch (LOGN_EXPR) { IBPF_CASES_512 default: break; }              \
  }

// ------------------------------------------------------------------ single-grid launches
// (allocation-free Poisson entry point, n <= 1024): block b takes the row pairs or the
// columns b * fft_per_block(n) ..
template <typename T>
__global__ void __launch_bounds__(kFftSmallThreads) k_rows_fwd(const T* __restrict__ in,
    typename C2T<T>::type* __restrict__ spec, int nx, int ny, int sp,
    const typename C2T<T>::type* __restrict__ tw) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  const int rp = fft_per_block(nx);
  const int cnt = min(rp, ny / 2 - (int)blockIdx.x * rp);
  const size_t ra = 2 * (size_t)blockIdx.x * rp;
#define IBPF_CASE(L) case L: rows_fwd_core<T, L, kFftSmallThreads>(in, spec, tw, ra, cnt, sp, x); break;
  switch (31 - __clz(nx)) { IBPF_CASES_128 default: break; }
#undef IBPF_CASE
}

template <typename T>
__global__ void __launch_bounds__(kFftSmallThreads) k_rows_inv(
    const typename C2T<T>::type* __restrict__ spec, T* out, int nx, int ny, int sp,
    const typename C2T<T>::type* __restrict__ tw, EpiArgs epi) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  const int rp = fft_per_block(nx);
  const int cnt = min(rp, ny / 2 - (int)blockIdx.x * rp);
  const size_t ra = 2 * (size_t)blockIdx.x * rp;
#define IBPF_CASE(L) case L: rows_inv_core<T, L, kFftSmallThreads>(spec, out, tw, epi, ra, cnt, sp, x); break;
  switch (31 - __clz(nx)) { IBPF_CASES_128 default: break; }
#undef IBPF_CASE
}

template <typename T>
__global__ void __launch_bounds__(kFftSmallThreads) k_cols(
    typename C2T<T>::type* __restrict__ spec, int nh1, int ny,
    const typename C2T<T>::type* __restrict__ tw, const typename C2T<T>::type* __restrict__ wd,
    SymbolArgs sym) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  const int k0 = blockIdx.x * fft_per_block(ny);
#define IBPF_CASE(L) case L: cols_core<T, L, kFftSmallThreads>(spec, nh1, tw, wd, sym, k0, x); break;
  switch (31 - __clz(ny)) { IBPF_CASES_128 default: break; }
#undef IBPF_CASE
}

// ------------------------------------------------------------------ batched launches
// One block per work unit (the grid is nblk blocks); THREADS selects the transform class.
// src: 0 the CH right-hand side Q, 1 the Poisson right-hand side, 2 / 3 the velocity
// predictor right-hand sides held in the u / v slot 1 - cur
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) kb_rows_fwd(const InstDev<T>* __restrict__ I,
    const int2* __restrict__ blk, int nblk, int src, int cur) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int2 w = blk[b];
  const InstDev<T>& d = I[w.x];
  const int rp = fft_per_block(d.nx);
  const int cnt = min(rp, d.ny / 2 - w.y * rp);
  const T* in = src == 0 ? d.Q : (src == 1 ? d.rhs : (src == 2 ? d.U[1 - cur] : d.V[1 - cur]));
  C2* x = reinterpret_cast<C2*>(smem_raw);
  const size_t ra = 2 * (size_t)w.y * rp;
#define IBPF_CASE(L) case L: rows_fwd_core<T, L, THREADS>(in, d.spec, d.twx, ra, cnt, d.nx / 2 + 1, x); break;
  IBPF_DISPATCH(THREADS, d.lognx)
#undef IBPF_CASE
}

template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) kb_cols(const InstDev<T>* __restrict__ I,
    const int2* __restrict__ blk, int nblk, int mode) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int2 w = blk[b];
  const InstDev<T>& d = I[w.x];
  SymbolArgs sym;
  sym.mode = mode;
  sym.s_eta2 = d.s_eta2;
  sym.c0 = d.c0;
  sym.s_eta2_f = (float)d.s_eta2;
  sym.c0_f = (float)d.c0;
  sym.lamx = d.lamx;
  sym.lamy = d.lamy;
  sym.lamx_f = d.lamx_f;
  sym.lamy_f = d.lamy_f;
  C2* x = reinterpret_cast<C2*>(smem_raw);
  const int nh1 = d.nx / 2 + 1, k0 = w.y * fft_per_block(d.ny);
#define IBPF_CASE(L) case L: cols_core<T, L, THREADS>(d.spec, nh1, d.twy, d.wd, sym, k0, x); break;
  IBPF_DISPATCH(THREADS, d.logny)
#undef IBPF_CASE
}

// the velocity Helmholtz solves of the semi-implicit predictor: (1 - a L) with the DST-II
// (u, no-slip ghost rows) and DST-I (v, zero wall faces) wall-normal bases
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) kb_cols_s2(const InstDev<T>* __restrict__ I,
    const int2* __restrict__ blk, int nblk) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int2 w = blk[b];
  const InstDev<T>& d = I[w.x];
  SymbolArgs sym;
  sym.mode = 2;
  sym.c0 = d.a_visc;
  sym.c0_f = (float)d.a_visc;
  sym.lamx = d.lamx;
  sym.lamy = d.lam_s2;
  sym.lamx_f = d.lamx_f;
  sym.lamy_f = d.lam_s2_f;
  C2* x = reinterpret_cast<C2*>(smem_raw);
  const int nh1 = d.nx / 2 + 1, k0 = w.y * fft_per_block(d.ny);
#define IBPF_CASE(L) case L: cols_core<T, L, THREADS, 8, true>(d.spec, nh1, d.twy, d.wd, sym, k0, x); break;
  IBPF_DISPATCH(THREADS, d.logny)
#undef IBPF_CASE
}

template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) kb_dst1(const InstDev<T>* __restrict__ I,
    const int2* __restrict__ blk, int nblk) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int2 w = blk[b];
  const InstDev<T>& d = I[w.x];
  SymbolArgs sym;
  sym.mode = 2;
  sym.c0 = d.a_visc;
  sym.c0_f = (float)d.a_visc;
  sym.lamx = d.lamx;
  sym.lamx_f = d.lamx_f;
  C2* x = reinterpret_cast<C2*>(smem_raw);
  const T* ld1 = sizeof(T) == 8 ? (const T*)d.lam_d1 : (const T*)d.lam_d1_f;
  const int nh1 = d.nx / 2 + 1, k0 = w.y * fft_per_block(2 * d.ny);
#define IBPF_CASE(L) case L: dst1_core<T, L, THREADS>(d.spec, nh1, d.tw2, sym, ld1, k0, x); break;
  IBPF_DISPATCH(THREADS, d.logny + 1)
#undef IBPF_CASE
}

// kind 1: C^{n+1} into the C^{n-1} slot (compensated in FP32); kind 2: P^{n+1} = P^ + dP;
// kind 3 / 4: the predicted velocity u** = alpha_u (u^n + du) / v** = alpha_v (v^n + dv)
// into the u / v slot 1 - cur (rows 0 .. ny-1)
template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS) kb_rows_inv(const InstDev<T>* __restrict__ I,
    const int2* __restrict__ blk, int nblk, int kind, int cur) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  if (b >= nblk) return;
  const int2 w = blk[b];
  const InstDev<T>& d = I[w.x];
  EpiArgs epi;
  epi.kind = kind;
  T* out;
  if (kind == 1) {
    epi.a = d.C[cur];
    epi.b = d.C[1 - cur];
    epi.a_lo = d.Clo[cur];
    epi.b_lo = d.Clo[1 - cur];
    epi.out_lo = d.Clo[1 - cur];
    out = d.C[1 - cur];
  } else if (kind == 2) {
    epi.a = d.phat;
    epi.delta = d.dp;
    out = d.P[1 - cur];
  } else {
    epi.kind = 3;
    epi.a = kind == 3 ? d.U[cur] : d.V[cur];
    epi.alpha = kind == 3 ? d.au : d.av;
    out = kind == 3 ? d.U[1 - cur] : d.V[1 - cur];
  }
  const int rp = fft_per_block(d.nx);
  const int cnt = min(rp, d.ny / 2 - w.y * rp);
  C2* x = reinterpret_cast<C2*>(smem_raw);
  const size_t ra = 2 * (size_t)w.y * rp;
#define IBPF_CASE(L) case L: rows_inv_core<T, L, THREADS>(d.spec, out, d.twx, epi, ra, cnt, d.nx / 2 + 1, x); break;
  IBPF_DISPATCH(THREADS, d.lognx)
#undef IBPF_CASE
}

// ------------------------------------------------------------------ 3D: strided axes
// The transforms along the strided axes of the 3D half spectrum spec[(z ny + y) sp + kx]
// (row pitch sp = nx/2 + 1 rounded up to even, so that every row starts on a 16-byte
// boundary; the pad column is zero from allocation on and stays zero) run on tiles of PW
// consecutive columns (one 128-byte segment per row: 16 FP32 or 8 FP64 complex values;
// 64 bytes for 1024-point transforms) times the whole transform length N.  One block per
// tile:
//   load   16-byte cp.async copies, consecutive threads on consecutive chunks of a row, all
//          issued before one wait: the whole tile is in flight at once and holds no
//          registers;
//   FFT    in place, radix 8 with one radix-2 or radix-4 pass for the rest of the length:
//          decimation in frequency forward, which leaves mode k at row fft_pos(k), and
//          decimation in time inverse, which takes that order back to natural order, so no
//          pass permutes;
//   store  the last pass writes its outputs from registers straight to global memory.
// A thread takes CP = 16 / sizeof(complex) adjacent columns of a butterfly (two in FP32,
// sharing its twiddles) with 16-byte shared-memory accesses; consecutive threads take
// consecutive column groups of a row, so no phase has bank conflicts.
// y axis: the forward transform leaves its rows in the order fft_pos (row p holds mode
// fft_rev(p)); the z solve takes the y eigenvalue of row p from a table in that order and
// the inverse y transform starts from it.

// mode held by row p after the forward passes of a 2^logn-point transform (radix-8 passes
// first): p's digits, most significant first, are the radix digits of the mode, least first
__host__ __device__ constexpr int fft_rev(int p, int logn) {
  int k = 0, lw = logn, lo = 0;
  while (lw > 0) {
    const int lr = lw >= 3 ? 3 : lw;
    lw -= lr;
    k |= ((p >> lw) & ((1 << lr) - 1)) << lo;
    lo += lr;
  }
  return k;
}
// row of mode k (the inverse of fft_rev)
__host__ __device__ constexpr int fft_pos(int k, int logn) {
  int p = 0, lw = logn, lo = 0;
  while (lw > 0) {
    const int lr = lw >= 3 ? 3 : lw;
    lw -= lr;
    p |= ((k >> lo) & ((1 << lr) - 1)) << lw;
    lo += lr;
  }
  return p;
}

constexpr int kTileThreads = 256;

// columns per tile of RB-byte rows (RB = 128: up to 512 points; RB = 64: from 256 points
// on, the only width for 1024 points, whose 128-byte tiles would leave one block per SM)
template <typename T, int RB>
__host__ __device__ constexpr int tile_cols() {
  return RB / (int)sizeof(typename C2T<T>::type);
}

// shared memory of a tile block: the tile, the twiddles (n), the cosine weights (n), the
// z eigenvalues (n) and the per-column eigenvalue parts (2 pw) (the last three: z solve)
template <typename T>
__host__ __device__ constexpr size_t tile_smem_bytes(int n, int pw, bool zsolve) {
  return sizeof(typename C2T<T>::type) * ((size_t)n * pw + n + (zsolve ? n : 0)) +
         (zsolve ? sizeof(T) * (n + 2 * pw) : 0);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}

// Rows rows(r) of the tile come from src + r * pitch (nc columns), in 16-byte chunks; the
// caller waits (cp.async.wait_all) and synchronises before reading them.  The copies need
// 16-byte aligned addresses and sizes: a tile whose source, pitch or width breaks that (no
// layout of this file does) is not loaded and false is returned to every thread.
template <int PW, int N, typename C2, typename RowMap>
__device__ __forceinline__ bool tile_load(C2* x, const C2* src, size_t pitch, int nc,
                                          RowMap rows) {
  const size_t bad = (reinterpret_cast<size_t>(src) | (pitch * sizeof(C2)) | (nc * sizeof(C2))) & 15;
  if (bad != 0 || nc <= 0 || nc > PW) return false;
  auto copy = [&](int r, int q) {
    cp_async16(reinterpret_cast<char*>(x + (size_t)rows(r) * PW) + 16 * q,
               reinterpret_cast<const char*>(src + r * pitch) + 16 * q);
  };
  constexpr int CPR = PW * (int)sizeof(C2) / 16;   // chunks of a full row
  if (nc == PW) {
#pragma unroll 4
    for (int c = threadIdx.x; c < N * CPR; c += kTileThreads) copy(c / CPR, c % CPR);
  } else {
    const int cpr = (int)(nc * sizeof(C2) / 16);
    for (int c = threadIdx.x; c < N * cpr; c += kTileThreads) copy(c / cpr, c % cpr);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  return true;
}
__device__ __forceinline__ void tile_wait() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
}

// the full twiddle table exp(-2 pi i t / N), t < N, in shared memory from the half table
// tw[m] = exp(-2 pi i m / N), m < N/2 (the other half is its negative)
template <int N, typename C2>
__device__ __forceinline__ void stage_twiddles(C2* tws, const C2* __restrict__ tw) {
  for (int t = threadIdx.x; t < N / 2; t += kTileThreads) {
    const C2 w = tw[t];
    tws[t] = w;
    tws[t + N / 2] = C2{-w.x, -w.y};
  }
}

// CP adjacent complex values of a tile row as one 16-byte shared-memory access
template <typename C2, int CP>
__device__ __forceinline__ void ld_cols(const C2* p, C2* v) {
  if constexpr (CP == 2) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0].x = q.x; v[0].y = q.y; v[1].x = q.z; v[1].y = q.w;
  } else {
    v[0] = *p;
  }
}
template <typename C2, int CP>
__device__ __forceinline__ void st_cols(C2* p, const C2* v) {
  if constexpr (CP == 2) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  } else {
    *p = v[0];
  }
}

// Pass S of the in-place transform of length N = 2^LOGN on the tile x (N rows of PW points):
// span L = N / 8^S, radix R = min(8, L), stride L/R.  Forward (decimation in frequency):
// v_r = x[b + j + r L/R], R-point DFT, output q times W_L^{j q}, back at b + j + q L/R.
// Inverse (decimation in time): the inverse of that step without its 1/R, input q times
// conj(W_L^{j q}), then the inverse R-point DFT.  A thread takes CP adjacent columns of a
// butterfly; put(row, column, values) takes every output (CP values from that column on).
template <int LOGN, int S, bool INV, int PW, typename T, typename C2, typename Put>
__device__ __forceinline__ void ip_pass(C2* x, const C2* __restrict__ tw, Put put) {
  constexpr int N = 1 << LOGN, LWB = LOGN - 3 * S;
  constexpr int LR = LWB >= 3 ? 3 : LWB, R = 1 << LR, L = 1 << LWB, STR = L / R;
  constexpr int CP = 16 / (int)sizeof(C2), NG = PW / CP;
  constexpr int NB = (N / R) * NG, TS = N / L;
#pragma unroll 2
  for (int u = threadIdx.x; u < NB; u += kTileThreads) {
    const int f = (u % NG) * CP, bf = u / NG;
    const int j = bf % STR, row0 = (bf / STR) * L + j;
    C2 v[CP][R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C2 t[CP];
      ld_cols<C2, CP>(x + (row0 + r * STR) * PW + f, t);
#pragma unroll
      for (int c = 0; c < CP; ++c) v[c][r] = t[c];
    }
    if constexpr (INV) {
      if constexpr (STR > 1) {
#pragma unroll
        for (int q = 1; q < R; ++q) {
          const C2 w = cconj(tw[j * q * TS]);
#pragma unroll
          for (int c = 0; c < CP; ++c) v[c][q] = cmul(v[c][q], w);
        }
      }
#pragma unroll
      for (int c = 0; c < CP; ++c) dft_reg<R, true, T>(v[c]);
    } else {
#pragma unroll
      for (int c = 0; c < CP; ++c) dft_reg<R, false, T>(v[c]);
      if constexpr (STR > 1) {
#pragma unroll
        for (int q = 1; q < R; ++q) {
          const C2 w = tw[j * q * TS];
#pragma unroll
          for (int c = 0; c < CP; ++c) v[c][q] = cmul(v[c][q], w);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C2 t[CP];
#pragma unroll
      for (int c = 0; c < CP; ++c) t[c] = v[c][r];
      put(row0 + r * STR, f, t);
    }
  }
}

// The whole in-place transform from pass K on: forward passes S = 0, 1, ..; inverse passes
// in the reverse order.  The last pass hands its outputs to `last`; the others store them
// back into the tile, with a barrier between passes.
template <int LOGN, int K, bool INV, int PW, typename T, typename C2, typename Put>
__device__ __forceinline__ void ip_fft(C2* x, const C2* __restrict__ tw, Put last) {
  constexpr int NP = (LOGN + 2) / 3;
  constexpr int S = INV ? NP - 1 - K : K;
  constexpr int CP = 16 / (int)sizeof(C2);
  if constexpr (K == NP - 1) {
    ip_pass<LOGN, S, INV, PW, T>(x, tw, last);
  } else {
    ip_pass<LOGN, S, INV, PW, T>(x, tw, [x](int row, int f, const C2* v) {
      st_cols<C2, CP>(x + row * PW + f, v);
    });
    __syncthreads();
    ip_fft<LOGN, K + 1, INV, PW, T>(x, tw, last);
  }
}

// CP values (columns f.. of a tile row) to global memory at p, scaled by sc, the columns at
// or beyond nc skipped (nc and f are multiples of CP)
template <typename C2, int CP, typename T>
__device__ __forceinline__ void st_global(C2* p, const C2* v, int f, int nc, T sc) {
  if (f >= nc) return;
  C2 o[CP];
#pragma unroll
  for (int c = 0; c < CP; ++c) {
    o[c].x = v[c].x * sc;
    o[c].y = v[c].y * sc;
  }
  st_cols<C2, CP>(p, o);
}

// y transform of one tile: z-plane blockIdx.x / nbt, columns kx0 = (blockIdx.x % nbt) PW ..
// (nc = min(PW, sp - kx0) of them).  Forward: rows in natural order in, in the order fft_pos
// out.  Inverse: back, scaled by 1/N.
template <typename T, int LOGN, bool INV, int RB>
__global__ void __launch_bounds__(kTileThreads) k3_ytile(typename C2T<T>::type* __restrict__ spec,
    int sp, int nbt, const typename C2T<T>::type* __restrict__ tw, int* status) {
  using C2 = typename C2T<T>::type;
  constexpr int N = 1 << LOGN, PW = tile_cols<T, RB>(), CP = 16 / (int)sizeof(C2);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  C2* tws = x + N * PW;
  const int z = blockIdx.x / nbt, kx0 = (int)(blockIdx.x % nbt) * PW;
  const int nc = min(PW, sp - kx0);
  C2* g = spec + (size_t)z * N * sp + kx0;
  if (!tile_load<PW, N>(x, g, (size_t)sp, nc, [](int r) { return r; })) {
    if (threadIdx.x == 0) atomicOr(status, 2);
    return;
  }
  stage_twiddles<N>(tws, tw);
  tile_wait();
  const T sc = INV ? T(1) / T(N) : T(1);
  ip_fft<LOGN, 0, INV, PW, T>(x, tws, [&](int row, int f, const C2* v) {
    st_global<C2, CP>(g + (size_t)row * sp + f, v, f, nc, sc);
  });
}

// z solve of one tile: columns k0 = blockIdx.x PW .. of the ny sp columns k = p sp + kx (p a y
// row in the order fft_pos).  Cosine transform along z by Makhoul's reordering (folded into
// the row copies: row r goes to r/2 if even, N - 1 - (r-1)/2 if odd) and an N-point FFT,
// division by the symbol at L = (lamz[m] + lamy[fft_rev(p)]) + lamx[kx], inverse transform
// and the inverse reordering on the way out (the pair formulas of cols_core).
template <typename T, int LOGN, int RB>
__global__ void __launch_bounds__(kTileThreads) k3_ztile(typename C2T<T>::type* __restrict__ spec,
    int ncols, int sp, int nh1, const typename C2T<T>::type* __restrict__ tw,
    const typename C2T<T>::type* __restrict__ wd, SymbolArgs sym, int* status) {
  using C2 = typename C2T<T>::type;
  constexpr int N = 1 << LOGN, PW = tile_cols<T, RB>(), half = N / 2;
  constexpr int CP = 16 / (int)sizeof(C2);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C2* x = reinterpret_cast<C2*>(smem_raw);
  C2* tws = x + N * PW;
  C2* wds = tws + N;
  T* lzs = reinterpret_cast<T*>(wds + N);   // lamz[m]
  T* lcx = lzs + N;                         // lamx[kx] of each column
  T* lcy = lcx + PW;                        // the y eigenvalue of each column's row
  const int k0 = blockIdx.x * PW;
  const int nc = min(PW, ncols - k0);
  const size_t pitch = (size_t)ncols;
  C2* g = spec + k0;
  if (!tile_load<PW, N>(x, g, pitch, nc,
                        [](int r) { return (r & 1) ? N - 1 - (r >> 1) : (r >> 1); })) {
    if (threadIdx.x == 0) atomicOr(status, 2);
    return;
  }
  const T* lamz = sizeof(T) == 8 ? (const T*)sym.lamy : (const T*)sym.lamy_f;
  const T* lam_x = sizeof(T) == 8 ? (const T*)sym.lamx : (const T*)sym.lamx_f;
  const T* lam_y = sizeof(T) == 8 ? (const T*)sym.lamyp : (const T*)sym.lamyp_f;
  stage_twiddles<N>(tws, tw);
  for (int t = threadIdx.x; t < N; t += kTileThreads) {
    wds[t] = wd[t];
    lzs[t] = lamz[t];
  }
  for (int c = threadIdx.x; c < PW; c += kTileThreads) {
    const int k = min(k0 + c, ncols - 1);
    lcx[c] = lam_x[min(k % sp, nh1 - 1)];   // the pad column (zero) takes the last mode's
    lcy[c] = lam_y[k / sp];
  }
  tile_wait();
  ip_fft<LOGN, 0, false, PW, T>(x, tws, [x](int row, int f, const C2* v) {
    st_cols<C2, CP>(x + row * PW + f, v);
  });
  __syncthreads();
  // pair tasks (m, N - m), m = 0..N/2, of CP adjacent columns; mode m sits at row fft_pos(m)
  constexpr int NG = PW / CP;
  for (int t = threadIdx.x; t < NG * (half + 1); t += kTileThreads) {
    const int c0 = (t % NG) * CP, m = t / NG;
    const int mm = (N - m) & (N - 1);
    C2* pm = x + fft_pos(m, LOGN) * PW + c0;
    C2* pmm = x + fft_pos(mm, LOGN) * PW + c0;
    C2 Vm[CP], Vmm[CP], Zm[CP], Zmm[CP];
    ld_cols<C2, CP>(pm, Vm);
    ld_cols<C2, CP>(pmm, Vmm);
    const C2 wm = wds[m], wmm = wds[mm];
    const T lzm = lzs[m], lzmm = lzs[mm];
#pragma unroll
    for (int c = 0; c < CP; ++c) {
      C2 Xm, Xmm;
      {
        C2 vr, vi;
        vr.x = T(0.5) * (Vm[c].x + Vmm[c].x);
        vr.y = T(0.5) * (Vm[c].y - Vmm[c].y);
        vi.x = T(0.5) * (Vm[c].y + Vmm[c].y);
        vi.y = T(-0.5) * (Vm[c].x - Vmm[c].x);
        Xm.x = wm.x * vr.x - wm.y * vr.y;
        Xm.y = wm.x * vi.x - wm.y * vi.y;
      }
      {
        C2 vr, vi;
        vr.x = T(0.5) * (Vmm[c].x + Vm[c].x);
        vr.y = T(0.5) * (Vmm[c].y - Vm[c].y);
        vi.x = T(0.5) * (Vmm[c].y + Vm[c].y);
        vi.y = T(-0.5) * (Vmm[c].x - Vm[c].x);
        Xmm.x = wmm.x * vr.x - wmm.y * vr.y;
        Xmm.y = wmm.x * vi.x - wmm.y * vi.y;
      }
      const T lc = lcy[c0 + c], lx = lcx[c0 + c];
      Xm = divide_symbol<T>(Xm, (lzm + lc) + lx, sym);
      Xmm = divide_symbol<T>(Xmm, (lzmm + lc) + lx, sym);
      {
        C2 y;   // X_m - i X_{N-m}; X_N = 0 for m = 0
        const C2 xo = (m == 0) ? C2{T(0), T(0)} : Xmm;
        y.x = Xm.x + xo.y;
        y.y = Xm.y - xo.x;
        Zm[c] = cmul(cconj(wm), y);
      }
      {
        C2 y;
        const C2 xo = (mm == 0) ? C2{T(0), T(0)} : Xm;
        y.x = Xmm.x + xo.y;
        y.y = Xmm.y - xo.x;
        Zmm[c] = cmul(cconj(wmm), y);
      }
    }
    st_cols<C2, CP>(pm, Zm);
    if (mm != m) st_cols<C2, CP>(pmm, Zmm);
  }
  __syncthreads();
  const T inv = T(1) / T(N);
  ip_fft<LOGN, 0, true, PW, T>(x, tws, [&](int n, int f, const C2* v) {
    const int r = n < half ? 2 * n : 2 * (N - 1 - n) + 1;
    st_global<C2, CP>(g + (size_t)r * pitch + f, v, f, nc, inv);
  });
}

// the row widths a tile transform of 2^logn points is built for
inline bool tile_rb_ok(int logn, int rb) {
  return (rb == 128 && logn <= 9) || (rb == 64 && logn >= 8);
}
// the default row width: 128 bytes up to 512 points, 64 bytes for 1024
inline int tile_rb_default(int logn) { return logn >= 10 ? 64 : 128; }

template <typename T, int L, int RB>
void tile_attributes_one() {
  const cudaFuncAttribute att = cudaFuncAttributeMaxDynamicSharedMemorySize;
  constexpr int PW = tile_cols<T, RB>();
  cudaFuncSetAttribute(k3_ytile<T, L, false, RB>, att, (int)tile_smem_bytes<T>(1 << L, PW, false));
  cudaFuncSetAttribute(k3_ytile<T, L, true, RB>, att, (int)tile_smem_bytes<T>(1 << L, PW, false));
  cudaFuncSetAttribute(k3_ztile<T, L, RB>, att, (int)tile_smem_bytes<T>(1 << L, PW, true));
}
// maximum dynamic shared memory of the tile kernels for lengths 2^L .. 2^10
template <typename T, int L>
void tile_attributes() {
  if constexpr (L <= 9) tile_attributes_one<T, L, 128>();
  if constexpr (L >= 8) tile_attributes_one<T, L, 64>();
  if constexpr (L < 10) tile_attributes<T, L + 1>();
}

#define IBPF_TILE_CASES IBPF_T(3, 128) IBPF_T(4, 128) IBPF_T(5, 128) IBPF_T(6, 128) IBPF_T(7, 128) \
  IBPF_T(8, 128) IBPF_T(9, 128) IBPF_T(8, 64) IBPF_T(9, 64) IBPF_T(10, 64)

template <typename T, bool INV>
void launch_ytile(int logn, int rb, int blocks, size_t smem, cudaStream_t s,
                  typename C2T<T>::type* spec, int sp, int nbt,
                  const typename C2T<T>::type* tw, int* status) {
#define IBPF_T(L, RB) \
  if (logn == L && rb == RB) k3_ytile<T, L, INV, RB><<<blocks, kTileThreads, smem, s>>>(spec, sp, nbt, tw, status);
  IBPF_TILE_CASES
#undef IBPF_T
}

template <typename T>
void launch_ztile(int logn, int rb, int blocks, size_t smem, cudaStream_t s,
                  typename C2T<T>::type* spec, int ncols, int sp, int nh1,
                  const typename C2T<T>::type* tw, const typename C2T<T>::type* wd,
                  const SymbolArgs& sym, int* status) {
#define IBPF_T(L, RB) \
  if (logn == L && rb == RB) k3_ztile<T, L, RB><<<blocks, kTileThreads, smem, s>>>(spec, ncols, sp, nh1, tw, wd, sym, status);
  IBPF_TILE_CASES
#undef IBPF_T
}

template <typename T>
cudaError_t tables_t(Instance& in) {
  using C2 = typename C2T<T>::type;
  const int nx = in.nx, ny = in.ny;
  const double h = in.h;
  std::vector<double> lx(nx / 2 + 1), ly(ny);
  for (int k = 0; k <= nx / 2; ++k) {
    double sn = std::sin(M_PI * (double)k / (double)nx);
    lx[k] = -(4.0 / (h * h)) * sn * sn;
  }
  for (int m = 0; m < ny; ++m) {
    double sn = std::sin(M_PI * (double)m / (2.0 * (double)ny));
    ly[m] = -(4.0 / (h * h)) * sn * sn;
  }
  std::vector<C2> twx(nx / 2), twy(ny / 2), wd(ny);
  for (int k = 0; k < nx / 2; ++k) {
    double a = 2.0 * M_PI * (double)k / (double)nx;
    twx[k].x = (T)std::cos(a);
    twx[k].y = (T)(-std::sin(a));
  }
  for (int k = 0; k < ny / 2; ++k) {
    double a = 2.0 * M_PI * (double)k / (double)ny;
    twy[k].x = (T)std::cos(a);
    twy[k].y = (T)(-std::sin(a));
  }
  for (int m = 0; m < ny; ++m) {
    double a = M_PI * (double)m / (2.0 * (double)ny);
    wd[m].x = (T)std::cos(a);
    wd[m].y = (T)(-std::sin(a));
  }
  cudaError_t e;
  if ((e = cudaMalloc((void**)&in.lamx, sizeof(double) * lx.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc((void**)&in.lamy, sizeof(double) * ly.size())) != cudaSuccess) return e;
  std::vector<float> lxf(lx.begin(), lx.end()), lyf(ly.begin(), ly.end());
  if ((e = cudaMalloc((void**)&in.lamx_f, sizeof(float) * lxf.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc((void**)&in.lamy_f, sizeof(float) * lyf.size())) != cudaSuccess) return e;
  cudaMemcpy(in.lamx_f, lxf.data(), sizeof(float) * lxf.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(in.lamy_f, lyf.data(), sizeof(float) * lyf.size(), cudaMemcpyHostToDevice);
  if ((e = cudaMalloc(&in.twx, sizeof(C2) * twx.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&in.twy, sizeof(C2) * twy.size())) != cudaSuccess) return e;
  if ((e = cudaMalloc(&in.wdct, sizeof(C2) * wd.size())) != cudaSuccess) return e;
  cudaMemcpy(in.lamx, lx.data(), sizeof(double) * lx.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(in.lamy, ly.data(), sizeof(double) * ly.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(in.twx, twx.data(), sizeof(C2) * twx.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(in.twy, twy.data(), sizeof(C2) * twy.size(), cudaMemcpyHostToDevice);
  e = cudaMemcpy(in.wdct, wd.data(), sizeof(C2) * wd.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  if (in.prm_ns_semi) {
    // semi-implicit predictor: DST-II eigenvalues in the cosine order k (mode m = ny - k),
    // DST-I eigenvalues of the modes 0 .. ny, twiddles of the 2 ny-point FFTs
    std::vector<double> ls2(ny), ld1(ny + 1);
    for (int k = 0; k < ny; ++k) {
      const double cs = std::cos(M_PI * (double)k / (2.0 * (double)ny));
      ls2[k] = -(4.0 / (h * h)) * cs * cs;
    }
    for (int m = 0; m <= ny; ++m) {
      const double sn = std::sin(M_PI * (double)m / (2.0 * (double)ny));
      ld1[m] = -(4.0 / (h * h)) * sn * sn;
    }
    std::vector<C2> tw2(ny);
    for (int k = 0; k < ny; ++k) {
      const double a = M_PI * (double)k / (double)ny;
      tw2[k].x = (T)std::cos(a);
      tw2[k].y = (T)(-std::sin(a));
    }
    std::vector<float> ls2f(ls2.begin(), ls2.end()), ld1f(ld1.begin(), ld1.end());
    if ((e = cudaMalloc((void**)&in.lam_s2, sizeof(double) * ls2.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&in.lam_d1, sizeof(double) * ld1.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&in.lam_s2_f, sizeof(float) * ls2f.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&in.lam_d1_f, sizeof(float) * ld1f.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc(&in.tw2, sizeof(C2) * tw2.size())) != cudaSuccess) return e;
    cudaMemcpy(in.lam_s2, ls2.data(), sizeof(double) * ls2.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(in.lam_d1, ld1.data(), sizeof(double) * ld1.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(in.lam_s2_f, ls2f.data(), sizeof(float) * ls2f.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(in.lam_d1_f, ld1f.data(), sizeof(float) * ld1f.size(), cudaMemcpyHostToDevice);
    e = cudaMemcpy(in.tw2, tw2.data(), sizeof(C2) * tw2.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  // the 4096-point class needs up to 120 KiB of shared memory (FP64)
  const int att = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaFuncSetAttribute(kb_rows_fwd<T, kFftSmallThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_rows_inv<T, kFftSmallThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_cols<T, kFftSmallThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_rows_fwd<T, kFftLargeThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_rows_inv<T, kFftLargeThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_cols<T, kFftLargeThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_cols_s2<T, kFftSmallThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_cols_s2<T, kFftLargeThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_dst1<T, kFftSmallThreads>, (cudaFuncAttribute)att, 200 * 1024);
  cudaFuncSetAttribute(kb_dst1<T, kFftLargeThreads>, (cudaFuncAttribute)att, 200 * 1024);
  return cudaGetLastError();
}

// 3D tables: lamx (nx/2+1, periodic x), lamy (ny, periodic y), lamz (nz, Neumann z) and the
// FP32 copies; twiddles of the x, y and z transforms and the z cosine weights
template <typename T>
cudaError_t tables3_t(Instance& in) {
  using C2 = typename C2T<T>::type;
  const int nx = in.nx, ny = in.ny, nz = in.nz;
  const double h = in.h;
  std::vector<double> lx(nx / 2 + 1), ly(ny), lz(nz);
  for (int k = 0; k <= nx / 2; ++k) {
    const double sn = std::sin(M_PI * (double)k / (double)nx);
    lx[k] = -(4.0 / (h * h)) * sn * sn;
  }
  // y eigenvalues in the row order of the y-transformed spectrum: row p holds mode
  // fft_rev(p) (the in-place forward transform leaves its modes in that order)
  int logny = 0;
  while ((1 << logny) < ny) ++logny;
  for (int p = 0; p < ny; ++p) {
    const double sn = std::sin(M_PI * (double)fft_rev(p, logny) / (double)ny);
    ly[p] = -(4.0 / (h * h)) * sn * sn;
  }
  for (int m = 0; m < nz; ++m) {
    const double sn = std::sin(M_PI * (double)m / (2.0 * (double)nz));
    lz[m] = -(4.0 / (h * h)) * sn * sn;
  }
  auto twiddles = [](int n) {
    std::vector<C2> t(n / 2);
    for (int k = 0; k < n / 2; ++k) {
      const double a = 2.0 * M_PI * (double)k / (double)n;
      t[k].x = (T)std::cos(a);
      t[k].y = (T)(-std::sin(a));
    }
    return t;
  };
  std::vector<C2> twx = twiddles(nx), twy = twiddles(ny), twz = twiddles(nz), wd(nz);
  for (int m = 0; m < nz; ++m) {
    const double a = M_PI * (double)m / (2.0 * (double)nz);
    wd[m].x = (T)std::cos(a);
    wd[m].y = (T)(-std::sin(a));
  }
  std::vector<float> lxf(lx.begin(), lx.end()), lyf(ly.begin(), ly.end()), lzf(lz.begin(), lz.end());
  cudaError_t e = cudaSuccess;
  auto put = [&](void** dst, const void* src, size_t bytes) {
    if ((e = cudaMalloc(dst, bytes)) != cudaSuccess) return false;
    return (e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice)) == cudaSuccess;
  };
  if (!put((void**)&in.lamx, lx.data(), sizeof(double) * lx.size()) ||
      !put((void**)&in.lamy, ly.data(), sizeof(double) * ly.size()) ||
      !put((void**)&in.lamz, lz.data(), sizeof(double) * lz.size()) ||
      !put((void**)&in.lamx_f, lxf.data(), sizeof(float) * lxf.size()) ||
      !put((void**)&in.lamy_f, lyf.data(), sizeof(float) * lyf.size()) ||
      !put((void**)&in.lamz_f, lzf.data(), sizeof(float) * lzf.size()) ||
      !put(&in.twx, twx.data(), sizeof(C2) * twx.size()) ||
      !put(&in.twy, twy.data(), sizeof(C2) * twy.size()) ||
      !put(&in.twz, twz.data(), sizeof(C2) * twz.size()) ||
      !put(&in.wdct, wd.data(), sizeof(C2) * wd.size()))
    return e;
  const cudaFuncAttribute att = cudaFuncAttributeMaxDynamicSharedMemorySize;
  (void)att;
  tile_attributes<T, 3>();
  if (in.tc_z && (e = zsolve_tc_tables(nz, &in.dmat_z)) != cudaSuccess) return e;

  return cudaGetLastError();
}

// row width of the instance's y / z tiles: the tuned one if set, else the default
inline int y_rb(const Instance& in) { return in.tune_y_rb ? in.tune_y_rb : tile_rb_default(in.logny); }
inline int z_rb(const Instance& in) { return in.tune_z_rb ? in.tune_z_rb : tile_rb_default(in.lognz); }

// the y transforms of a 3D spectrum (forward or inverse) with rb-byte tile rows
template <typename T>
void ytile3(const Instance& in, bool inv, int rb, cudaStream_t s) {
  using C2 = typename C2T<T>::type;
  const int sp = spec3_pitch(in.nx);
  const int pw = rb / (int)sizeof(C2), nbt = (sp + pw - 1) / pw;
  const size_t sm = tile_smem_bytes<T>(in.ny, pw, false);
  if (inv) launch_ytile<T, true>(in.logny, rb, in.nz * nbt, sm, s, (C2*)in.spec, sp, nbt, (const C2*)in.twy, in.status);
  else launch_ytile<T, false>(in.logny, rb, in.nz * nbt, sm, s, (C2*)in.spec, sp, nbt, (const C2*)in.twy, in.status);
}

// the z solve of a 3D spectrum (mode 0: CH symbol, 1: Poisson) with rb-byte tile rows
template <typename T>
void ztile3(const Instance& in, int mode, int rb, cudaStream_t s) {
  using C2 = typename C2T<T>::type;
  const int nh1 = in.nx / 2 + 1, sp = spec3_pitch(in.nx);
  SymbolArgs sym;
  sym.mode = mode;
  sym.s_eta2 = in.prm.S / (in.prm.Cn * in.prm.Cn);
  sym.c0 = 1.5 * in.prm.Pe / (in.prm.Cn * in.prm.Cn * in.prm.dt);
  sym.s_eta2_f = (float)sym.s_eta2;
  sym.c0_f = (float)sym.c0;
  sym.lamx = in.lamx;
  sym.lamy = in.lamz;
  sym.lamx_f = in.lamx_f;
  sym.lamy_f = in.lamz_f;
  sym.ncx = nh1;
  sym.lamyp = in.lamy;
  sym.lamyp_f = in.lamy_f;
  const int ncols = in.ny * sp, pw = rb / (int)sizeof(C2);
  launch_ztile<T>(in.lognz, rb, (ncols + pw - 1) / pw, tile_smem_bytes<T>(in.nz, pw, true), s,
                  (C2*)in.spec, ncols, sp, nh1, (const C2*)in.twz, (const C2*)in.wdct, sym, in.status);
}

// One 3D solve: x rows, y columns, z cosine transform + symbol + inverse, y inverse, x rows
// inverse with the epilogue of the batched 2D solve (mode 0: C increment into the C^{n-1}
// slot, compensated in FP32; mode 1: P^{n+1} = P^ + dP).
template <typename T>
int spectral3_solve_t(const Instance& in, int mode, int cur, cudaStream_t s, Recorder* rec) {
  using C2 = typename C2T<T>::type;
  constexpr int S = kFftSmallThreads;
  const int nx = in.nx, ny = in.ny, nz = in.nz, sp = spec3_pitch(nx);
  const int rows = ny * nz;
  const int rp = fft_per_block(nx);
  C2* spec = (C2*)in.spec;
  // the row kernels take at most 26 KiB of shared memory; the tile kernels up to 88 KiB,
  // allowed by the attributes set with the tables
  const size_t rsm = sizeof(C2) * (fft_buf(8 * S) + nx / 2);
  const T* src = (const T*)(mode == 0 ? in.Q : in.rhs);
  k_rows_fwd<T><<<(rows / 2 + rp - 1) / rp, S, rsm, s>>>(src, spec, nx, rows, sp, (const C2*)in.twx);
  if (rec) rec->mark("rows_fwd", s);
  ytile3<T>(in, false, y_rb(in), s);
  if (rec) rec->mark("y_fft", s);
  if (in.tc_z && sizeof(T) == 4) {
    zsolve_tc_launch((float*)in.spec, nz, (long long)ny * sp, sp, nx / 2 + 1, in.lamz_f, in.lamx_f,
                     in.lamy_f, in.dmat_z, mode, (float)(in.prm.S / (in.prm.Cn * in.prm.Cn)),
                     (float)(1.5 * in.prm.Pe / (in.prm.Cn * in.prm.Cn * in.prm.dt)), in.status, s);
    if (rec) rec->mark("z_solve_tc", s);
  } else {
    ztile3<T>(in, mode, z_rb(in), s);
    if (rec) rec->mark("z_solve", s);
  }
  ytile3<T>(in, true, y_rb(in), s);
  if (rec) rec->mark("y_ifft", s);
  EpiArgs epi;
  T* out;
  if (mode == 0) {
    epi.kind = 1;
    epi.a = in.C[cur];
    epi.b = in.C[1 - cur];
    epi.a_lo = in.Clo[cur];
    epi.b_lo = in.Clo[1 - cur];
    epi.out_lo = in.Clo[1 - cur];
    out = (T*)in.C[1 - cur];
  } else {
    epi.kind = 2;
    epi.a = in.phat;
    epi.delta = in.dp;
    out = (T*)in.P[1 - cur];
  }
  k_rows_inv<T><<<(rows / 2 + rp - 1) / rp, S, rsm, s>>>(spec, out, nx, rows, sp, (const C2*)in.twx, epi);
  if (rec) rec->mark("rows_inv", s);
  return 5;
}

}  // namespace

template <typename T>
int spectral_solve_batch(const BatchPlan& plan, int mode, int cur, cudaStream_t s,
                         Recorder* rec) {
  // mode 0: Cahn-Hilliard (Q -> C^{n+1}), 1: Poisson (rhs -> P^{n+1}), 2 / 3: the semi-implicit
  // predictor's u / v Helmholtz solves (dt F in the u** slot -> u** = alpha (u^n + d))
  const InstDev<T>* I = reinterpret_cast<const InstDev<T>*>(plan.d_inst);
  constexpr int S = kFftSmallThreads, L = kFftLargeThreads;
  const int kind = mode == 0 ? 1 : (mode == 1 ? 2 : (mode == 2 ? 3 : 4));
  const char* cname = mode == 2 ? "vel_cols_u" : (mode == 3 ? "vel_cols_v" : "cols_solve");
  const char* fname = mode >= 2 ? "vel_rows_fwd" : "rows_fwd";
  const char* iname = mode >= 2 ? "vel_rows_inv" : "rows_inv";
  int n = 0;
  if (plan.nblk[kFamRows]) {
    kb_rows_fwd<T, S><<<plan.nblk[kFamRows], S, plan.rows_smem[0], s>>>(
        I, plan.d_blk[kFamRows], plan.nblk[kFamRows], mode, cur);
    if (rec) rec->mark(fname, s);
    ++n;
  }
  if (plan.nblk[kFamRowsL]) {
    kb_rows_fwd<T, L><<<plan.nblk[kFamRowsL], L, plan.rows_smem[1], s>>>(
        I, plan.d_blk[kFamRowsL], plan.nblk[kFamRowsL], mode, cur);
    if (rec) rec->mark(fname, s);
    ++n;
  }
  if (mode <= 2) {
    for (int c = 0; c < 2; ++c) {
      const int f = c ? kFamColsL : kFamCols;
      if (!plan.nblk[f]) continue;
      if (mode == 2) {
        if (c) kb_cols_s2<T, L><<<plan.nblk[f], L, plan.cols_smem[1], s>>>(I, plan.d_blk[f], plan.nblk[f]);
        else kb_cols_s2<T, S><<<plan.nblk[f], S, plan.cols_smem[0], s>>>(I, plan.d_blk[f], plan.nblk[f]);
      } else {
        if (c) kb_cols<T, L><<<plan.nblk[f], L, plan.cols_smem[1], s>>>(I, plan.d_blk[f], plan.nblk[f], mode);
        else kb_cols<T, S><<<plan.nblk[f], S, plan.cols_smem[0], s>>>(I, plan.d_blk[f], plan.nblk[f], mode);
      }
      if (rec) rec->mark(cname, s);
      ++n;
    }
  } else {
    for (int c = 0; c < 2; ++c) {
      const int f = c ? kFamD1L : kFamD1;
      if (!plan.nblk[f]) continue;
      if (c) kb_dst1<T, L><<<plan.nblk[f], L, plan.d1_smem[1], s>>>(I, plan.d_blk[f], plan.nblk[f]);
      else kb_dst1<T, S><<<plan.nblk[f], S, plan.d1_smem[0], s>>>(I, plan.d_blk[f], plan.nblk[f]);
      if (rec) rec->mark(cname, s);
      ++n;
    }
  }
  if (plan.nblk[kFamRows]) {
    kb_rows_inv<T, S><<<plan.nblk[kFamRows], S, plan.rows_smem[0], s>>>(
        I, plan.d_blk[kFamRows], plan.nblk[kFamRows], kind, cur);
    if (rec) rec->mark(iname, s);
    ++n;
  }
  if (plan.nblk[kFamRowsL]) {
    kb_rows_inv<T, L><<<plan.nblk[kFamRowsL], L, plan.rows_smem[1], s>>>(
        I, plan.d_blk[kFamRowsL], plan.nblk[kFamRowsL], kind, cur);
    if (rec) rec->mark(iname, s);
    ++n;
  }
  return n;
}
template int spectral_solve_batch<double>(const BatchPlan&, int, int, cudaStream_t, Recorder*);
template int spectral_solve_batch<float>(const BatchPlan&, int, int, cudaStream_t, Recorder*);

int spectral_solve_ptrs(int nx, int ny, const double* rhs, double* out, int mode, double s_eta2,
                        double c0, double2* spec, const double* lamx, const double* lamy,
                        const double2* twx, const double2* twy, const double2* wd,
                        cudaStream_t s) {
  const int nh1 = nx / 2 + 1;
  const int rp = fft_per_block(nx), cp = fft_per_block(ny);
  constexpr int S = kFftSmallThreads;
  // nx, ny <= 1024 here: the row buffers take at most 26 KiB and the column buffers 42 KiB
  // of shared memory, below the default limit, so this path sets no function attributes
  const size_t rsm = sizeof(double2) * (fft_buf(8 * S) + nx / 2);
  const size_t csm = cols_smem_bytes<double>(ny, 8 * S);
  k_rows_fwd<double><<<(ny / 2 + rp - 1) / rp, S, rsm, s>>>(rhs, spec, nx, ny, nh1, twx);
  SymbolArgs sym;
  sym.mode = mode;
  sym.s_eta2 = s_eta2;
  sym.c0 = c0;
  sym.lamx = lamx;
  sym.lamy = lamy;
  k_cols<double><<<(nh1 + cp - 1) / cp, S, csm, s>>>(spec, nh1, ny, twy, wd, sym);
  EpiArgs plain;
  k_rows_inv<double><<<(ny / 2 + rp - 1) / rp, S, rsm, s>>>(spec, out, nx, ny, nh1, twx, plain);
  return 3;
}

cudaError_t spectral3_tables(Instance& in, int precision) {
  return precision == IB_PF_FP64 ? tables3_t<double>(in) : tables3_t<float>(in);
}

// Tuner: the mean time (ms) of `reps` launches of the y transforms (axis 1: forward and
// inverse, halved) or of the z solve (axis 2, Poisson symbol) with rb-byte tile rows, run on
// the instance's spectral scratch (whose content every solve overwrites).  -1: rb is not
// built for that length.
float spectral3_time_tiles(const Instance& in, int precision, int axis, int rb, int reps,
                           cudaStream_t s) {
  const int logn = axis == 1 ? in.logny : in.lognz;
  if (!tile_rb_ok(logn, rb)) return -1.0f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto once = [&]() {
    if (precision == IB_PF_FP64) {
      if (axis == 1) { ytile3<double>(in, false, rb, s); ytile3<double>(in, true, rb, s); }
      else ztile3<double>(in, 1, rb, s);
    } else {
      if (axis == 1) { ytile3<float>(in, false, rb, s); ytile3<float>(in, true, rb, s); }
      else ztile3<float>(in, 1, rb, s);
    }
  };
  once();   // warm-up
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) once();
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / (float)reps / (axis == 1 ? 2.0f : 1.0f);
}

int spectral3_solve(const Instance& in, int precision, int mode, int cur, cudaStream_t s,
                    Recorder* rec) {
  return precision == IB_PF_FP64 ? spectral3_solve_t<double>(in, mode, cur, s, rec)
                                 : spectral3_solve_t<float>(in, mode, cur, s, rec);
}

cudaError_t spectral_tables(Instance& in, int precision) {
  return precision == IB_PF_FP64 ? tables_t<double>(in) : tables_t<float>(in);
}

}  // namespace ibpf
