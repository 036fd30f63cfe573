// Wall-normal (z) solve of a 3D spectrum on the tensor cores, in split-BF16 products
// (precision IB_PF_FP32_3XBF16; Appendix A.1 and Eq. PressurePoisson).
//
// The solve of the separable operator along the wall-normal axis is, per spectral column
// (kx, ky) of length N = nz:  x <- D^T diag(1 / sigma(kx, ky, m)) D x,  with D the orthonormal
// DCT-II, D[m][z] = c_m cos(pi m (2z + 1) / (2N)), c_0 = sqrt(1/N), c_m = sqrt(2/N) (the
// eigenvectors of the zero-gradient second difference, Sec. 4.4 and Appendix A.1), sigma the
// symbol of the Cahn-Hilliard split (L^2 - (S/Cn^2) L + 1.5 Pe/(Cn^2 dt)) or the Poisson
// operator (L, zero mode set to 0), L = lamz[m] + lamy[ky] + lamx[kx].
//
// Both transforms are dense matrix products on the tensor cores.  N = 256 takes one even/odd
// (radix-2) step first, which halves the products: with u_j = x_j + x_{N-1-j},
// v_j = x_j - x_{N-1-j} (j < N/2),  X_{2p} = (Ce u)_p and X_{2p+1} = (Co v)_p, where
// Ce[p][j] = D[2p][j] and Co[p][j] = D[2p+1][j]; the inverse is a = Ce^T Y_even,
// b = Co^T Y_odd, x_j = a_j + b_j, x_{N-1-j} = a_j - b_j (D[2p][N-1-j] = D[2p][j],
// D[2p+1][N-1-j] = -D[2p+1][j]).  N = 128 uses D itself.  Every product is then
// 128 x 128, H = N / 128 of them per transform.
//
// Split precision: every FP32 operand value x is held as hi + lo with hi = bf16(x),
// lo = bf16(x - hi) (16 significant bits); a product is accumulated in FP32 tensor memory as
// Ahi Bhi + Alo Bhi + Ahi Blo (the Alo Blo term, ~2^-16 relative, is dropped).  The matrices
// are rounded once from FP64 on the host.
//
// Kernel layout: persistent, one block of 512 threads per SM.  The H x {hi, lo} matrices
// (H x 64 KiB) arrive once per block by bulk copies and stay in shared memory as the B
// operands: K-major for the forward products, the same bytes read MN-major for the inverse.
// A tile is 128 real spectrum columns (64 complex) of all N rows, with the columns on the
// tensor-memory lanes (MMA M = 128, N = 128):
//   forward  D1[n][m] = sum_j X[n][j] Mat[m][j], X the tile after the even/odd step, split
//            and written to tensor memory as the A operand;
//   symbol   Z[n][m] = D1[n][m] / sigma, split, written over X as the next A operand;
//   inverse  D2[n][j] = sum_m Z[n][m] Mat[m][j], the even/odd step undone on the way out.
// Each thread owns one column (its lane) and a quarter of the rows, so a warp's loads and
// stores touch 32 consecutive floats of a spectrum row.  The next tile's loads are issued
// under the forward and the inverse products.

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "ibpf_internal.h"
#include "tc_ptx.cuh"

namespace ibpf {
namespace {

constexpr int kTcMat = 128 * 128 * 2;          // bytes of one 128 x 128 BF16 matrix

// Matrix layout in shared memory: element (m, j) (row m of Ce, Co or D, column j) at
// ((m/8) 16 + j/8) 128 + (m%8) 16 + (j%8) 2, core matrices of 8 rows of 16 bytes.  As the B
// operand of the forward products (K = j, N = m) that is K-major: K-adjacent core matrices
// 128 bytes apart (LBO), N-adjacent 2048 (SBO); of the inverse ones (K = m, N = j) MN-major:
// K-adjacent 2048 (LBO), N-adjacent 128 (SBO).
constexpr uint32_t kA_LBO_K = 128, kA_SBO_K = 2048;
constexpr uint32_t kA_LBO_MN = 2048, kA_SBO_MN = 128;

__host__ __device__ constexpr int a_off(int m, int k) {
  return (((m >> 3) * 16 + (k >> 3)) << 7) + ((m & 7) << 4) + ((k & 7) << 1);
}

struct TcZArgs {
  float* spec;           // nz rows of 2 ncols floats (complex spectrum, interleaved re/im)
  long long ncols;       // complex columns per z row (ny x sp)
  int sp, nh1;           // spectrum row pitch in complex values, x modes nx/2 + 1
  const float* lamz;     // nz wall-normal eigenvalues, natural mode order
  const float* lamx;     // nh1
  const float* lamyp;    // ny: y eigenvalue of each spectrum row (the order the y FFT left)
  const void* dmat;      // H x {hi, lo} matrices in the shared-memory layout
  int mode;              // 0: Cahn-Hilliard symbol, 1: Poisson
  float s_eta2, c0;      // S / Cn^2, 1.5 Pe / (Cn^2 dt), rounded once
  int* status;           // bit 4: a bounded wait gave up
};

// a, b -> their BF16 parts (hi and lo, two per 32-bit word, a in the low half)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
constexpr int kTtThreads = 512;
constexpr int kTtCols = 128;          // real columns per tile
constexpr uint32_t kTtXA = 0;         // tensor-memory columns of the A operands: (2h + part) 64
constexpr uint32_t kTtD = 256;        // accumulators: h 128

template <int H>
struct TtSmem {
  static constexpr int A = 0;                      // H x {hi, lo} matrices
  static constexpr int LZ = A + 2 * H * kTcMat;    // lamz (N floats)
  static constexpr int BAR = LZ + 4 * 128 * H;     // 3 mbarriers, tensor-memory base, flag
  static constexpr int BYTES = BAR + 64;
};

// one thread's share of a tile: column n, rows j = 32 sub + i (i < 32) and N - 1 - j
template <int H>
struct TtRegs {
  float x[32];
  float y[32];
  float lc;      // lamy + lamx of the column's complex mode
};

// rows i in [I0, I0 + 16) of this thread's share (the lc term with the first half)
template <int H, int I0>
__device__ __forceinline__ void tt_load(TtRegs<H>& r, const TcZArgs& a, size_t pitch, long long c0, int ncr,
                                        int n, int sub) {
  constexpr int N = 128 * H;
  const bool in = n < ncr;
  if constexpr (I0 == 0) {
    const long long kc = min((c0 + n) / 2, a.ncols - 1);
    r.lc = a.lamyp[kc / a.sp] + a.lamx[min((int)(kc % a.sp), a.nh1 - 1)];
  }
  const float* col = a.spec + c0 + n;
#pragma unroll
  for (int i = I0; i < I0 + 16; ++i) {
    const int j = 32 * sub + i;
    r.x[i] = in ? col[(size_t)j * pitch] : 0.f;
    if constexpr (H == 2) r.y[i] = in ? col[(size_t)(N - 1 - j) * pitch] : 0.f;
  }
}

// the even/odd step (H = 2) and the split of the forward A operands into tensor memory
template <int H>
__device__ __forceinline__ void tt_store_x(const TtRegs<H>& r, uint32_t t_lane, int sub) {
  uint32_t hi[16], lo[16];
  if constexpr (H == 2) {
#pragma unroll
    for (int i = 0; i < 16; ++i) split2(r.x[2 * i] + r.y[2 * i], r.x[2 * i + 1] + r.y[2 * i + 1], hi[i], lo[i]);
    tc::tmem_st16(t_lane + kTtXA + 0 * 64 + 16 * sub, hi);
    tc::tmem_st16(t_lane + kTtXA + 1 * 64 + 16 * sub, lo);
#pragma unroll
    for (int i = 0; i < 16; ++i) split2(r.x[2 * i] - r.y[2 * i], r.x[2 * i + 1] - r.y[2 * i + 1], hi[i], lo[i]);
    tc::tmem_st16(t_lane + kTtXA + 2 * 64 + 16 * sub, hi);
    tc::tmem_st16(t_lane + kTtXA + 3 * 64 + 16 * sub, lo);
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) split2(r.x[2 * i], r.x[2 * i + 1], hi[i], lo[i]);
    tc::tmem_st16(t_lane + kTtXA + 0 * 64 + 16 * sub, hi);
    tc::tmem_st16(t_lane + kTtXA + 1 * 64 + 16 * sub, lo);
  }
}

template <int H, bool FWD>
__device__ __forceinline__ void tt_products(uint32_t sa, uint32_t tmem) {
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 128, false, !FWD);
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const uint32_t m_hi = sa + (2 * h) * kTcMat, m_lo = m_hi + kTcMat;
    const uint32_t a_hi = tmem + kTtXA + (2 * h) * 64, a_lo = a_hi + 64;
    const uint32_t d = tmem + kTtD + h * 128;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const uint32_t bo = FWD ? s * 256 : s * 4096;
      const uint32_t lbo = FWD ? kA_LBO_K : kA_LBO_MN, sbo = FWD ? kA_SBO_K : kA_SBO_MN;
      const uint64_t bh = tc::sdesc(m_hi + bo, lbo, sbo), bl = tc::sdesc(m_lo + bo, lbo, sbo);
      tc::mma_bf16_ts(d, a_hi + 8 * s, bl, idesc, s > 0 ? 1u : 0u);
      tc::mma_bf16_ts(d, a_lo + 8 * s, bh, idesc, 1u);
      tc::mma_bf16_ts(d, a_hi + 8 * s, bh, idesc, 1u);
    }
  }
}

template <int H>
__global__ void __launch_bounds__(kTtThreads, 1) k3_zsolve_tt(TcZArgs a) {
  using L = TtSmem<H>;
  constexpr int N = 128 * H, NT = kTtCols;
  extern __shared__ __align__(1024) unsigned char sm[];
  float* s_lz = reinterpret_cast<float*>(sm + L::LZ);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);   // matrices, forward, inverse
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + L::BAR + 24);
  int* s_abort = reinterpret_cast<int*>(sm + L::BAR + 28);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q = warp & 3, sub = warp >> 2, n = 32 * q + lane;
  const uint32_t sa = tc::smem_u32(sm + L::A);

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) tc::mbar_init(&bar[i], 1);
    tc::mbar_init_fence();
    *s_abort = 0;
  }
  for (int m = tid; m < N; m += kTtThreads) s_lz[m] = a.lamz[m];
  __syncthreads();
  if (tid == 0) {
    constexpr uint32_t bytes = 2u * H * kTcMat;
    tc::mbar_expect_tx(&bar[0], bytes);
    for (uint32_t off = 0; off < bytes; off += 16384)
      tc::bulk_g2s(sm + L::A + off, static_cast<const unsigned char*>(a.dmat) + off, 16384, &bar[0]);
  }
  __syncwarp();
  if (warp == 0) tc::tmem_alloc(s_tmem, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;
  const uint32_t t_lane = tmem + ((uint32_t)(32 * q) << 16);
  if (tid == 0 && !tc::mbar_wait(&bar[0], 0)) {
    *s_abort = 1;
    atomicOr(a.status, 4);
  }
  const long long ncr_all = 2 * a.ncols;
  const size_t pitch = (size_t)ncr_all;
  const long long ntiles = (ncr_all + NT - 1) / NT;
  auto tile_cols = [&](long long t) { return (int)min((long long)NT, ncr_all - t * NT); };

  TtRegs<H> r;
  long long t = blockIdx.x;
  if (t < ntiles) {
    tt_load<H, 0>(r, a, pitch, t * NT, tile_cols(t), n, sub);
    tt_load<H, 16>(r, a, pitch, t * NT, tile_cols(t), n, sub);
  }
  for (int k = 0; t < ntiles; ++k, t += gridDim.x) {
    const long long c0 = t * NT;
    const int ncr = tile_cols(t);
    const float lc = r.lc;
    tt_store_x<H>(r, t_lane, sub);
    tc::tmem_st_wait();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (*s_abort) break;
    if (tid == 0) {
      tt_products<H, true>(sa, tmem);
      tc::mma_commit(&bar[1]);
    }
    __syncwarp();
    // the next tile's loads, half now (under the forward products), half under the inverse
    const long long tn = t + gridDim.x;
    if (tn < ntiles) tt_load<H, 0>(r, a, pitch, tn * NT, tile_cols(tn), n, sub);
    if (!tc::mbar_wait(&bar[1], k & 1)) {
      *s_abort = 1;
      atomicOr(a.status, 4);
    }
    tc::fence_after_sync();
    // divide by the symbol: the quotients become the inverse A operands (over the forward ones)
#pragma unroll
    for (int h = 0; h < H; ++h) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float v[16];
        tc::tmem_ld16(t_lane + kTtD + h * 128 + 32 * sub + 16 * c, v);
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float z[2];
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int m = 32 * sub + 16 * c + 2 * i + e;
            const float Lv = s_lz[H == 2 ? 2 * m + h : m] + lc;
            float rr;
            if (a.mode == 0) rr = __fdividef(1.0f, (Lv - a.s_eta2) * Lv + a.c0);
            else rr = (Lv == 0.0f) ? 0.0f : __fdividef(1.0f, Lv);
            z[e] = v[2 * i + e] * rr;
          }
          split2(z[0], z[1], hi[i], lo[i]);
        }
        tc::tmem_st8(t_lane + kTtXA + (2 * h) * 64 + 16 * sub + 8 * c, hi);
        tc::tmem_st8(t_lane + kTtXA + (2 * h + 1) * 64 + 16 * sub + 8 * c, lo);
      }
    }
    tc::tmem_st_wait();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (*s_abort) break;
    if (tid == 0) {
      tt_products<H, false>(sa, tmem);
      tc::mma_commit(&bar[2]);
    }
    __syncwarp();
    if (tn < ntiles) tt_load<H, 16>(r, a, pitch, tn * NT, tile_cols(tn), n, sub);
    if (!tc::mbar_wait(&bar[2], k & 1)) {
      *s_abort = 1;
      atomicOr(a.status, 4);
    }
    tc::fence_after_sync();
    // undo the even/odd step; a warp stores 32 consecutive floats of a row
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float ya[16], yb[16];
      tc::tmem_ld16(t_lane + kTtD + 32 * sub + 16 * c, ya);
      if constexpr (H == 2) tc::tmem_ld16(t_lane + kTtD + 128 + 32 * sub + 16 * c, yb);
      if (n < ncr) {
        float* col = a.spec + c0 + n;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int j = 32 * sub + 16 * c + i;
          if constexpr (H == 2) {
            col[(size_t)j * pitch] = ya[i] + yb[i];
            col[(size_t)(N - 1 - j) * pitch] = ya[i] - yb[i];
          } else {
            col[(size_t)j * pitch] = ya[i];
          }
        }
      }
    }
    tc::fence_before_sync();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}


uint16_t bf16_bits(float f) {   // round to nearest even (finite inputs)
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

bool zsolve_tc_supported(int nz) { return nz == 128 || nz == 256; }

// the H x {hi, lo} matrices of an nz-point z solve (nz = 128 or 256), device copy in *out
cudaError_t zsolve_tc_tables(int nz, void** out) {
  const int H = nz / 128;
  std::vector<uint16_t> buf((size_t)2 * H * kTcMat / 2, 0);
  const double n = (double)nz;
  for (int h = 0; h < H; ++h)
    for (int p = 0; p < 128; ++p) {
      const int m = H == 2 ? 2 * p + h : p;
      const double cm = m == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
      for (int j = 0; j < 128; ++j) {
        const double d = cm * std::cos(M_PI * (double)m * (2.0 * j + 1.0) / (2.0 * n));
        const uint16_t hb = bf16_bits((float)d);
        const uint16_t lb = bf16_bits((float)(d - (double)bf16_value(hb)));
        const size_t o = (size_t)a_off(p, j) / 2;
        buf[(size_t)(2 * h) * (kTcMat / 2) + o] = hb;
        buf[(size_t)(2 * h + 1) * (kTcMat / 2) + o] = lb;
      }
    }
  cudaError_t e = cudaMalloc(out, buf.size() * 2);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*out, buf.data(), buf.size() * 2, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k3_zsolve_tt<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TtSmem<1>::BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k3_zsolve_tt<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TtSmem<2>::BYTES);
}

// the z solve of a 3D FP32 spectrum: spec holds nz rows of ncols complex values
void zsolve_tc_launch(float* spec, int nz, long long ncols, int sp, int nh1, const float* lamz,
                      const float* lamx, const float* lamyp, const void* dmat, int mode, float s_eta2,
                      float c0, int* status, cudaStream_t s) {
  TcZArgs a;
  a.spec = spec;
  a.ncols = ncols;
  a.sp = sp;
  a.nh1 = nh1;
  a.lamz = lamz;
  a.lamx = lamx;
  a.lamyp = lamyp;
  a.dmat = dmat;
  a.mode = mode;
  a.s_eta2 = s_eta2;
  a.c0 = c0;
  a.status = status;
  const long long tiles = (2 * ncols + kTtCols - 1) / kTtCols;
  const int grid = (int)std::min<long long>(tiles, sm_count());
  if (nz == 256) k3_zsolve_tt<2><<<grid, kTtThreads, TtSmem<2>::BYTES, s>>>(a);
  else k3_zsolve_tt<1><<<grid, kTtThreads, TtSmem<1>::BYTES, s>>>(a);
}

}  // namespace ibpf
