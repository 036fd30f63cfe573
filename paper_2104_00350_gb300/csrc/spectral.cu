// Separable spectral solves of the hybrid IB / phase-field step (Appendix A.1 and
// Eq. PressurePoisson): the 5-point Laplacian with periodic x1 and zero-gradient x2 walls
// is diagonal in the basis  exp(2 pi i k x1 / Lx)  x  cos(pi m (j + 1/2) / ny).
//
// A solve is three kernels:
//   rows_fwd : real FFT of every x1 row (two rows packed into one complex FFT),
//   cols     : per spectral column k, cosine transform (DCT-II) along x2, division by the
//              symbol in FP64, inverse cosine transform (the last forward axis and the first
//              inverse axis fused in shared memory),
//   rows_inv : inverse real FFT of every row (two rows per complex FFT).
// FFTs are radix-2 in shared memory: decimation in time on bit-reversed input for the
// forward transforms, decimation in frequency to bit-reversed output for the inverse ones.
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

__device__ __forceinline__ int brev(int n, int logn) {
  return logn == 0 ? 0 : (int)(__brev((unsigned)n) >> (32 - logn));
}

// cnt independent in-place radix-2 FFTs of length N = 2^logn stored back to back in x;
// every thread of the block takes butterflies of all of them, so one barrier per stage
// serves cnt transforms.
// DIT: input in bit-reversed order, output natural; tw[k] = exp(-2 pi i k/N), k < N/2.
template <typename C2>
__device__ void fft_dit(C2* x, int logn, const C2* __restrict__ tw, int cnt) {
  const int N = 1 << logn, half = N >> 1;
  for (int s = 0; s < logn; ++s) {
    const int m = 1 << s;
    const int tstride = N >> (s + 1);
    for (int t = threadIdx.x; t < cnt * half; t += blockDim.x) {
      const int f = t >> (logn - 1), p = t & (half - 1);
      C2* y = x + f * N;
      const int pos = p & (m - 1);
      const int i0 = ((p >> s) << (s + 1)) + pos;
      const int i1 = i0 + m;
      C2 b = cmul(tw[pos * tstride], y[i1]);
      C2 a = y[i0];
      y[i0] = cadd(a, b);
      y[i1] = csub(a, b);
    }
    __syncthreads();
  }
}

// DIF inverse without the 1/N: input natural, output bit-reversed, twiddles exp(+2 pi i k/N).
template <typename C2>
__device__ void ifft_dif(C2* x, int logn, const C2* __restrict__ tw, int cnt) {
  const int N = 1 << logn, half = N >> 1;
  for (int s = logn - 1; s >= 0; --s) {
    const int m = 1 << s;
    const int tstride = N >> (s + 1);
    for (int t = threadIdx.x; t < cnt * half; t += blockDim.x) {
      const int f = t >> (logn - 1), p = t & (half - 1);
      C2* y = x + f * N;
      const int pos = p & (m - 1);
      const int i0 = ((p >> s) << (s + 1)) + pos;
      const int i1 = i0 + m;
      C2 a = y[i0], b = y[i1];
      y[i0] = cadd(a, b);
      y[i1] = cmul(cconj(tw[pos * tstride]), csub(a, b));
    }
    __syncthreads();
  }
}

// Forward real FFT of the cnt row pairs (ra + 2f, ra + 2f + 1), f < cnt, of in (ny x nx)
// into spec (ny x (nx/2+1)).  Per pair z = row_a + i row_b;
// A_k = (Z_k + conj Z_{N-k})/2,  B_k = (Z_k - conj Z_{N-k})/(2i).
template <typename T>
__device__ void rows_fwd_core(const T* __restrict__ in, typename C2T<T>::type* __restrict__ spec,
                              int lognx, const typename C2T<T>::type* __restrict__ tw,
                              size_t ra, int cnt, typename C2T<T>::type* x) {
  using C2 = typename C2T<T>::type;
  const int nx = 1 << lognx, nh = nx >> 1;
  C2* tws = x + cnt * nx;   // twiddles staged after the data
  for (int t = threadIdx.x; t < nh; t += blockDim.x) tws[t] = tw[t];
  for (int t = threadIdx.x; t < cnt * nx; t += blockDim.x) {
    const int f = t >> lognx, n = t & (nx - 1);
    const size_t r = ra + 2 * f;
    C2 z;
    z.x = in[r * nx + n];
    z.y = in[(r + 1) * nx + n];
    x[f * nx + brev(n, lognx)] = z;
  }
  __syncthreads();
  fft_dit(x, lognx, tws, cnt);
  for (int t = threadIdx.x; t < cnt * (nh + 1); t += blockDim.x) {
    const int f = t / (nh + 1), k = t - f * (nh + 1);
    const C2* y = x + f * nx;
    const size_t r = ra + 2 * f;
    C2 z = y[k & (nx - 1)], zc = y[(nx - k) & (nx - 1)];
    C2 A, B;
    A.x = T(0.5) * (z.x + zc.x);
    A.y = T(0.5) * (z.y - zc.y);
    B.x = T(0.5) * (z.y + zc.y);
    B.y = T(-0.5) * (z.x - zc.x);
    spec[r * (nh + 1) + k] = A;
    spec[(r + 1) * (nh + 1) + k] = B;
  }
  __syncthreads();   // the shared buffer may be reused by the caller
}

template <typename T>
__global__ void k_rows_fwd(const T* __restrict__ in, typename C2T<T>::type* __restrict__ spec,
                           int lognx, const typename C2T<T>::type* __restrict__ tw) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_fwd_core<T>(in, spec, lognx, tw, 2 * (size_t)blockIdx.x, 1, reinterpret_cast<C2*>(smem_raw));
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

// Inverse of k_rows_fwd: Z_k = A_k + i B_k with Hermitian extension (imaginary parts of
// the k = 0 and k = nx/2 bins dropped), z = IFFT(Z)/nx, row_a = Re z, row_b = Im z.
// Epilogue (the solves return increments):
//   kind 0: out = z
//   kind 1: out = a + ((a - b)/3 + z)    (BDF2 predictor (2a - b/2)/1.5 of C plus the
//                                          increment, small terms first; out may alias b)
//   kind 2: delta = z, out = z + a         (pressure increment on top of a = P^)
template <typename T>
__device__ void rows_inv_core(const typename C2T<T>::type* __restrict__ spec, T* out, int lognx,
                              const typename C2T<T>::type* __restrict__ tw, const EpiArgs& epi,
                              size_t ra, int cnt, typename C2T<T>::type* x) {
  using C2 = typename C2T<T>::type;
  const int nx = 1 << lognx, nh = nx >> 1;
  for (int t = threadIdx.x; t < cnt * nx; t += blockDim.x) {
    const int f = t >> lognx, k = t & (nx - 1);
    const size_t r = ra + 2 * f;
    int kk = k <= nh ? k : nx - k;
    C2 A = spec[r * (nh + 1) + kk], B = spec[(r + 1) * (nh + 1) + kk];
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
    x[f * nx + k] = z;
  }
  C2* tws = x + cnt * nx;   // twiddles staged after the data
  for (int t = threadIdx.x; t < nh; t += blockDim.x) tws[t] = tw[t];
  __syncthreads();
  ifft_dif(x, lognx, tws, cnt);
  const T inv = T(1) / T(nx);
  const T* ea = reinterpret_cast<const T*>(epi.a);
  const T* eb = reinterpret_cast<const T*>(epi.b);
  T* ed = reinterpret_cast<T*>(epi.delta);
  for (int t = threadIdx.x; t < cnt * nx; t += blockDim.x) {
    const int f = t >> lognx, n = t & (nx - 1);
    const size_t r = ra + 2 * f;
    C2 z = x[f * nx + brev(n, lognx)];
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
    }
    out[ia] = va;
    out[ib] = vb;
  }
  __syncthreads();
}

template <typename T>
__global__ void k_rows_inv(const typename C2T<T>::type* __restrict__ spec, T* out, int lognx,
                           const typename C2T<T>::type* __restrict__ tw, EpiArgs epi) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rows_inv_core<T>(spec, out, lognx, tw, epi, 2 * (size_t)blockIdx.x, 1, reinterpret_cast<C2*>(smem_raw));
}

struct SymbolArgs {
  int mode;          // 0: Cahn-Hilliard quartic, 1: Poisson
  double s_eta2;     // S / Cn^2
  double c0;         // 1.5 Pe / (Cn^2 dt)
  const double* lamx;
  const double* lamy;
  const float* lamx_f;   // FP32 path: eigenvalues computed in FP64, rounded once
  const float* lamy_f;
};

// Divide X_m by the symbol at (k, m).  FP64 path: in FP64.  FP32 path: in FP32 -- the
// three terms of L^2 - (S/Cn^2) L + c0 (L <= 0) and the two of L are all of one sign, so
// the FP32 evaluation has no cancellation and keeps FP32 relative accuracy (FP64 here
// would occupy GB300's narrow FP64 pipe for most of the kernel).
template <typename T, typename C2>
__device__ __forceinline__ C2 divide_symbol(C2 X, int k, int m, const SymbolArgs& sym) {
  if constexpr (sizeof(T) == 8) {
    const double L = sym.lamy[m] + sym.lamx[k];
    if (sym.mode == 0) {
      const double sg = L * L - sym.s_eta2 * L + sym.c0;
      X.x = (T)((double)X.x / sg);
      X.y = (T)((double)X.y / sg);
    } else if (L == 0.0) {
      X.x = T(0);
      X.y = T(0);
    } else {
      X.x = (T)((double)X.x / L);
      X.y = (T)((double)X.y / L);
    }
  } else {
    const float L = sym.lamy_f[m] + sym.lamx_f[k];
    float r;
    if (sym.mode == 0) r = 1.0f / (L * L - (float)sym.s_eta2 * L + (float)sym.c0);
    else r = (L == 0.0f) ? 0.0f : 1.0f / L;
    X.x = X.x * r;
    X.y = X.y * r;
  }
  return X;
}

// x2 cosine transform, symbol division and inverse cosine transform of KC spectral
// columns per block (complex data; the transform is real so it acts on Re and Im alike).
//   forward  X_m = sum_j x_j cos(pi m (2j+1)/(2N)) via V = FFT(v), v the even/odd reorder:
//            X_m = Re(w_m Vr_m) + i Re(w_m Vi_m), w_m = exp(-i pi m/(2N)),
//            Vr_m = (V_m + conj V_{N-m})/2, Vi_m = (V_m - conj V_{N-m})/(2i);
//   divide   X_m /= sigma(k, m) in FP64;
//   inverse  Z_m = conj(w_m) (X_m - i X_{N-m}) (X_N = 0), z = IFFT(Z)/N,
//            x_{2n} = z_n, x_{2n+1} = z_{N-1-n}.
template <typename T, int KC>
__device__ void cols_core(typename C2T<T>::type* __restrict__ spec, int nh1, int logny,
                          const typename C2T<T>::type* __restrict__ tw,
                          const typename C2T<T>::type* __restrict__ wd, const SymbolArgs& sym,
                          int k0, typename C2T<T>::type* xs) {
  using C2 = typename C2T<T>::type;
  const int N = 1 << logny, half = N >> 1;
  C2* tws = xs + KC * N;     // FFT twiddles, staged once per block
  C2* wds = tws + half;      // cosine-transform weights
  for (int t = threadIdx.x; t < half; t += blockDim.x) tws[t] = tw[t];
  for (int t = threadIdx.x; t < N; t += blockDim.x) wds[t] = wd[t];
  // load: consecutive threads take consecutive columns of one row (coalesced)
  for (int idx = threadIdx.x; idx < KC * N; idx += blockDim.x) {
    int cc = idx % KC, r = idx / KC;
    int k = k0 + cc;
    C2 val;
    val.x = T(0);
    val.y = T(0);
    if (k < nh1) val = spec[(size_t)r * nh1 + k];
    int pos = (r & 1) ? (N - 1 - (r >> 1)) : (r >> 1);
    xs[cc * N + brev(pos, logny)] = val;
  }
  __syncthreads();
  fft_dit(xs, logny, tws, KC);
  // pair tasks (m, N - m), m = 0..N/2, of every column
  for (int t = threadIdx.x; t < KC * (half + 1); t += blockDim.x) {
    const int c = t / (half + 1), m = t - c * (half + 1);
    C2* x = xs + c * N;
    const int k = min(k0 + c, nh1 - 1);
    const int mm = (N - m) & (N - 1);
    C2 Vm = x[m], Vmm = x[mm];
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
    Xm = divide_symbol<T>(Xm, k, m, sym);
    Xmm = divide_symbol<T>(Xmm, k, mm, sym);
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
    x[m] = Zm;
    if (mm != m) x[mm] = Zmm;
  }
  __syncthreads();
  ifft_dif(xs, logny, tws, KC);
  const T inv = T(1) / T(N);
  for (int idx = threadIdx.x; idx < KC * N; idx += blockDim.x) {
    int cc = idx % KC, r = idx / KC;
    int kk = k0 + cc;
    int n = (r & 1) ? (N - 1 - (r >> 1)) : (r >> 1);
    C2 z = xs[cc * N + brev(n, logny)];
    z.x *= inv;
    z.y *= inv;
    if (kk < nh1) spec[(size_t)r * nh1 + kk] = z;
  }
  __syncthreads();
}

template <typename T, int KC>
__global__ void k_cols(typename C2T<T>::type* __restrict__ spec, int nh1, int logny,
                       const typename C2T<T>::type* __restrict__ tw,
                       const typename C2T<T>::type* __restrict__ wd, SymbolArgs sym) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cols_core<T, KC>(spec, nh1, logny, tw, wd, sym, blockIdx.x * KC, reinterpret_cast<C2*>(smem_raw));
}

// ------------------------------------------------------------------ batched launches
template <typename T>
__global__ void kb_rows_fwd(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                            int nblk, int src) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int2 w = blk[b];
    const InstDev<T>& d = I[w.x];
    const int cnt = min(kRowPairs, d.ny / 2 - w.y * kRowPairs);
    rows_fwd_core<T>(src == 0 ? d.Q : d.rhs, d.spec, d.lognx, d.twx, 2 * (size_t)w.y * kRowPairs,
                     cnt, reinterpret_cast<C2*>(smem_raw));
  }
}

template <typename T>
__global__ void kb_cols(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk, int nblk,
                        int mode) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int2 w = blk[b];
    const InstDev<T>& d = I[w.x];
    SymbolArgs sym;
    sym.mode = mode;
    sym.s_eta2 = d.s_eta2;
    sym.c0 = d.c0;
    sym.lamx = d.lamx;
    sym.lamy = d.lamy;
    sym.lamx_f = d.lamx_f;
    sym.lamy_f = d.lamy_f;
    cols_core<T, kColsKC>(d.spec, d.nx / 2 + 1, d.logny, d.twy, d.wd, sym, w.y * kColsKC,
                          reinterpret_cast<C2*>(smem_raw));
  }
}

// kind 1: C^{n+1} into the C^{n-1} slot (compensated in FP32); kind 2: P^{n+1} = P^ + dP
template <typename T>
__global__ void kb_rows_inv(const InstDev<T>* __restrict__ I, const int2* __restrict__ blk,
                            int nblk, int kind, int cur) {
  using C2 = typename C2T<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
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
    } else {
      epi.a = d.phat;
      epi.delta = d.dp;
      out = d.P[1 - cur];
    }
    const int cnt = min(kRowPairs, d.ny / 2 - w.y * kRowPairs);
    rows_inv_core<T>(d.spec, out, d.lognx, d.twx, epi, 2 * (size_t)w.y * kRowPairs, cnt,
                     reinterpret_cast<C2*>(smem_raw));
  }
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
  // rows of up to 4096 points need 64 KiB of shared memory (FP64)
  cudaFuncSetAttribute(kb_rows_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(kb_rows_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(kb_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
int spectral_solve_batch(const BatchPlan& plan, int mode, int cur, cudaStream_t s,
                         Recorder* rec) {
  const InstDev<T>* I = reinterpret_cast<const InstDev<T>*>(plan.d_inst);
  kb_rows_fwd<T><<<plan.nblk[kFamRows], plan.rows_threads, plan.rows_smem, s>>>(
      I, plan.d_blk[kFamRows], plan.nblk[kFamRows], mode);
  if (rec) rec->mark("rows_fwd", s);
  kb_cols<T><<<plan.nblk[kFamCols], plan.cols_threads, plan.cols_smem, s>>>(
      I, plan.d_blk[kFamCols], plan.nblk[kFamCols], mode);
  if (rec) rec->mark("cols_solve", s);
  kb_rows_inv<T><<<plan.nblk[kFamRows], plan.rows_threads, plan.rows_smem, s>>>(
      I, plan.d_blk[kFamRows], plan.nblk[kFamRows], mode == 0 ? 1 : 2, cur);
  if (rec) rec->mark("rows_inv", s);
  return 3;
}
template int spectral_solve_batch<double>(const BatchPlan&, int, int, cudaStream_t, Recorder*);
template int spectral_solve_batch<float>(const BatchPlan&, int, int, cudaStream_t, Recorder*);

int spectral_solve_ptrs(int nx, int ny, const double* rhs, double* out, int mode, double s_eta2,
                        double c0, double2* spec, const double* lamx, const double* lamy,
                        const double2* twx, const double2* twy, const double2* wd,
                        cudaStream_t s) {
  int lognx = 0, logny = 0;
  while ((1 << lognx) < nx) ++lognx;
  while ((1 << logny) < ny) ++logny;
  const int nh1 = nx / 2 + 1;
  const int trow = nx / 2 < 512 ? nx / 2 : 512;
  k_rows_fwd<double><<<ny / 2, trow, sizeof(double2) * (nx + nx / 2), s>>>(rhs, spec, lognx, twx);
  SymbolArgs sym;
  sym.mode = mode;
  sym.s_eta2 = s_eta2;
  sym.c0 = c0;
  sym.lamx = lamx;
  sym.lamy = lamy;
  // one column per block: data, twiddles and weights take at most 40 KiB of shared memory
  // for ny <= 1024, below the default limit, so this path needs no function attributes
  k_cols<double, 1><<<nh1, 256, sizeof(double2) * (ny + ny / 2 + ny), s>>>(spec, nh1, logny, twy,
                                                                         wd, sym);
  EpiArgs plain;
  k_rows_inv<double><<<ny / 2, trow, sizeof(double2) * (nx + nx / 2), s>>>(spec, out, lognx, twx,
                                                                           plain);
  return 3;
}

cudaError_t spectral_tables(Instance& in, int precision) {
  return precision == IB_PF_FP64 ? tables_t<double>(in) : tables_t<float>(in);
}

}  // namespace ibpf
