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
// 128 x 128 (one MMA tile height), H = N / 128 of them per transform.
//
// Split precision: every FP32 operand value x is held as hi + lo with hi = bf16(x),
// lo = bf16(x - hi) (16 significant bits); a product is accumulated in FP32 tensor memory as
// Ahi Bhi + Ahi Blo + Alo Bhi (the Alo Blo term, ~2^-16 relative, is dropped).  The matrices
// are rounded once from FP64 on the host.
//
// Kernel layout: persistent, one block of 256 threads per SM.  The H x {hi, lo} matrices
// (H x 64 KiB) arrive once per block by bulk copies and stay in shared memory; the same
// bytes serve the forward product (K-major A) and the inverse one (the transpose, read as an
// MN-major A).  A tile is 64 real columns (32 complex spectrum columns) of all N rows: loaded
// from global memory with the even/odd step applied, split, stored as the MN-major B operand;
// one thread issues the forward MMAs into tensor memory (H x 64 FP32 columns); the epilogue
// reads the accumulators, divides by the symbol, splits the result into the B operand of the
// inverse products; the inverse MMAs reuse the same tensor-memory columns; the last epilogue
// undoes the even/odd step and stores the columns.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "ibpf_internal.h"
#include "tc_ptx.cuh"

namespace ibpf {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcNG = 64;                      // real columns per tile (MMA N)
constexpr int kTcMat = 128 * 128 * 2;          // bytes of one 128 x 128 BF16 matrix
constexpr int kTcOpB = 128 * kTcNG * 2;        // bytes of one 128 x NG BF16 B operand

// descriptor strides (bytes) of the two layouts, see tc_ptx.cuh
//   matrices (A): K-major, element (m, k) at ((m/8) 16 + k/8) 128 + (m%8) 16 + (k%8) 2
//   tiles (B):    MN-major, element (k, n) at ((k/8) (NG/8) + n/8) 128 + (k%8) 16 + (n%8) 2
constexpr uint32_t kA_LBO_K = 128, kA_SBO_K = 2048;     // forward: K-major
constexpr uint32_t kA_LBO_MN = 2048, kA_SBO_MN = 128;   // inverse: the transpose, MN-major
constexpr uint32_t kB_LBO = kTcNG * 16, kB_SBO = 128;   // MN-major

__host__ __device__ constexpr int a_off(int m, int k) {
  return (((m >> 3) * 16 + (k >> 3)) << 7) + ((m & 7) << 4) + ((k & 7) << 1);
}
__host__ __device__ constexpr int b_off(int k, int n) {
  return (((k >> 3) * (kTcNG / 8) + (n >> 3)) << 7) + ((k & 7) << 4) + ((n & 7) << 1);
}

template <int H>
struct TcSmem {
  static constexpr int A = 0;                                   // H x {hi, lo} matrices
  static constexpr int B = A + 2 * H * kTcMat;                   // H x {hi, lo} tiles
  static constexpr int LZ = B + 2 * H * kTcOpB;                  // lamz (N floats)
  static constexpr int LC = LZ + 4 * 128 * H;                    // lamy + lamx of the tile's
  static constexpr int BAR = LC + 4 * (kTcNG / 2);               //   complex columns; barriers
  static constexpr int BYTES = BAR + 64;
};

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
// 8 values -> 16 bytes of hi parts and 16 bytes of lo parts
__device__ __forceinline__ void split8(const float* x, uint4& hi, uint4& lo) {
  split2(x[0], x[1], hi.x, lo.x);
  split2(x[2], x[3], hi.y, lo.y);
  split2(x[4], x[5], hi.z, lo.z);
  split2(x[6], x[7], hi.w, lo.w);
}

// forward (FWD) or inverse products of one tile: for each of the H matrices, 8 K-steps of
// 3 split MMAs into the tensor-memory columns tmem + h NG .. + NG - 1
template <int H, bool FWD>
__device__ __forceinline__ void issue_products(uint32_t sa, uint32_t sb, uint32_t tmem) {
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, kTcNG, !FWD, true);
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const uint32_t a_hi = sa + (2 * h) * kTcMat, a_lo = a_hi + kTcMat;
    const uint32_t b_hi = sb + (2 * h) * kTcOpB, b_lo = b_hi + kTcOpB;
    const uint32_t d = tmem + h * kTcNG;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const uint32_t ao = FWD ? s * 256 : s * 4096;   // K-step of 16: two core matrices
      const uint32_t lbo = FWD ? kA_LBO_K : kA_LBO_MN, sbo = FWD ? kA_SBO_K : kA_SBO_MN;
      const uint32_t bo = s * 2 * kB_LBO;
      const uint64_t ah = tc::sdesc(a_hi + ao, lbo, sbo), al = tc::sdesc(a_lo + ao, lbo, sbo);
      const uint64_t bh = tc::sdesc(b_hi + bo, kB_LBO, kB_SBO), bl = tc::sdesc(b_lo + bo, kB_LBO, kB_SBO);
      tc::mma_bf16(d, ah, bl, idesc, s > 0 ? 1u : 0u);
      tc::mma_bf16(d, al, bh, idesc, 1u);
      tc::mma_bf16(d, ah, bh, idesc, 1u);
    }
  }
}

// This thread's share of a tile: rows j = 8 ((warp >> 1) + 4 i) + (lane & 7), i < 4, and (for
// H = 2) N - 1 - j; real columns 8 g .. 8 g + 7, g = (lane >> 3) + 4 (warp & 1).
template <int H>
struct TileRegs {
  float4 x[4][2];
  float4 y[4][2];   // rows N - 1 - j (H = 2)
  float lc;         // threads 0..NG/2-1: lamy + lamx of complex column tid of the tile
};

template <int H>
__device__ __forceinline__ void load_tile(TileRegs<H>& r, const TcZArgs& a, size_t pitch, long long c0,
                                          int ncr, int warp, int lane) {
  constexpr int N = 128 * H;
  const float* spec = a.spec;
  if (threadIdx.x < kTcNG / 2) {
    const long long kc = min(c0 / 2 + threadIdx.x, a.ncols - 1);
    r.lc = a.lamyp[kc / a.sp] + a.lamx[min((int)(kc % a.sp), a.nh1 - 1)];
  }
  const int col = 8 * ((lane >> 3) + 4 * (warp & 1));
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = 8 * ((warp >> 1) + 4 * i) + (lane & 7);
    const float* r0 = spec + (size_t)j * pitch + c0 + col;
    r.x[i][0] = col < ncr ? *reinterpret_cast<const float4*>(r0) : z4;
    r.x[i][1] = col + 4 < ncr ? *reinterpret_cast<const float4*>(r0 + 4) : z4;
    if constexpr (H == 2) {
      const float* r1 = spec + (size_t)(N - 1 - j) * pitch + c0 + col;
      r.y[i][0] = col < ncr ? *reinterpret_cast<const float4*>(r1) : z4;
      r.y[i][1] = col + 4 < ncr ? *reinterpret_cast<const float4*>(r1 + 4) : z4;
    }
  }
}

// the even/odd step (H = 2), the split, and the stores of the forward B operands
template <int H>
__device__ __forceinline__ void store_tile(const TileRegs<H>& r, unsigned char* bt, int warp, int lane) {
  const int col = 8 * ((lane >> 3) + 4 * (warp & 1));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = 8 * ((warp >> 1) + 4 * i) + (lane & 7);
    const float x0[8] = {r.x[i][0].x, r.x[i][0].y, r.x[i][0].z, r.x[i][0].w,
                         r.x[i][1].x, r.x[i][1].y, r.x[i][1].z, r.x[i][1].w};
    const int o = b_off(j, col);
    uint4 hi, lo;
    if constexpr (H == 2) {
      const float x1[8] = {r.y[i][0].x, r.y[i][0].y, r.y[i][0].z, r.y[i][0].w,
                           r.y[i][1].x, r.y[i][1].y, r.y[i][1].z, r.y[i][1].w};
      float u[8], v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        u[e] = x0[e] + x1[e];
        v[e] = x0[e] - x1[e];
      }
      split8(u, hi, lo);
      *reinterpret_cast<uint4*>(bt + o) = hi;
      *reinterpret_cast<uint4*>(bt + kTcOpB + o) = lo;
      split8(v, hi, lo);
      *reinterpret_cast<uint4*>(bt + 2 * kTcOpB + o) = hi;
      *reinterpret_cast<uint4*>(bt + 3 * kTcOpB + o) = lo;
    } else {
      split8(x0, hi, lo);
      *reinterpret_cast<uint4*>(bt + o) = hi;
      *reinterpret_cast<uint4*>(bt + kTcOpB + o) = lo;
    }
  }
}

// the inverse products' results of a tile (tensor-memory columns tcol): undo the even/odd
// step and store this thread's 32 columns of row j (and N - 1 - j)
template <int H>
__device__ __forceinline__ void store_result(float* spec, size_t pitch, long long c0, int ncr,
                                             uint32_t t_row, int lq, int ch, int lane) {
  constexpr int N = 128 * H, NG = kTcNG;
  const int j = 32 * lq + lane, n0 = 32 * ch;
  float ya[32], yb[32];
  tc::tmem_ld32(t_row, ya);
  if constexpr (H == 2) tc::tmem_ld32(t_row + NG, yb);
  if (n0 >= ncr) return;
  float* o0 = spec + (size_t)j * pitch + c0 + n0;
  float* o1 = spec + (size_t)(N - 1 - j) * pitch + c0 + n0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (n0 + 4 * q < ncr) {
      if constexpr (H == 2) {
        *reinterpret_cast<float4*>(o0 + 4 * q) =
            make_float4(ya[4 * q] + yb[4 * q], ya[4 * q + 1] + yb[4 * q + 1], ya[4 * q + 2] + yb[4 * q + 2],
                        ya[4 * q + 3] + yb[4 * q + 3]);
        *reinterpret_cast<float4*>(o1 + 4 * q) =
            make_float4(ya[4 * q] - yb[4 * q], ya[4 * q + 1] - yb[4 * q + 1], ya[4 * q + 2] - yb[4 * q + 2],
                        ya[4 * q + 3] - yb[4 * q + 3]);
      } else {
        *reinterpret_cast<float4*>(o0 + 4 * q) = make_float4(ya[4 * q], ya[4 * q + 1], ya[4 * q + 2], ya[4 * q + 3]);
      }
    }
  }
}

// Software pipeline over the block's tiles t_0, t_1, ... (tensor memory holds two sets of
// accumulators, k & 1 for tile t_k):  store t_k's operands (loaded into registers during the
// previous tile) | forward MMAs of t_k, meanwhile the stores of t_{k-1} and the loads of
// t_{k+1} | symbol division | inverse MMAs of t_k.
template <int H>
__global__ void __launch_bounds__(kTcThreads, 1) k3_zsolve_tc(TcZArgs a) {
  using L = TcSmem<H>;
  constexpr int N = 128 * H, NG = kTcNG, NGC = NG / 2;
  extern __shared__ __align__(1024) unsigned char sm[];
  float* s_lz = reinterpret_cast<float*>(sm + L::LZ);
  float* s_lc = reinterpret_cast<float*>(sm + L::LC);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);   // matrices, forward, inverse
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + L::BAR + 24);
  int* s_abort = reinterpret_cast<int*>(sm + L::BAR + 28);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sa = tc::smem_u32(sm + L::A), sb = tc::smem_u32(sm + L::B);
  unsigned char* const bt = sm + L::B;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) tc::mbar_init(&bar[i], 1);
    tc::mbar_init_fence();
    *s_abort = 0;
  }
  for (int m = tid; m < N; m += kTcThreads) s_lz[m] = a.lamz[m];
  __syncthreads();
  if (tid == 0) {
    constexpr uint32_t bytes = 2u * H * kTcMat;
    tc::mbar_expect_tx(&bar[0], bytes);
    for (uint32_t off = 0; off < bytes; off += 16384)
      tc::bulk_g2s(sm + L::A + off, static_cast<const unsigned char*>(a.dmat) + off, 16384, &bar[0]);
  }
  __syncwarp();
  if (warp == 0) tc::tmem_alloc(s_tmem, 2 * H * NG);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *s_tmem;
  if (tid == 0 && !tc::mbar_wait(&bar[0], 0)) {
    *s_abort = 1;
    atomicOr(a.status, 4);
  }
  const long long ncr_all = 2 * a.ncols;      // real columns
  const size_t pitch = (size_t)ncr_all;       // floats per z row
  const long long ntiles = (ncr_all + NG - 1) / NG;
  const int lq = warp & 3, ch = warp >> 2;    // tensor-memory lane quarter, 32-column half
  const uint32_t t_lane = tmem + ((uint32_t)(32 * lq) << 16) + 32 * ch;
  auto tile_cols = [&](long long t) { return (int)min((long long)NG, ncr_all - t * NG); };

  TileRegs<H> regs;
  long long t = blockIdx.x;
  if (t < ntiles) load_tile<H>(regs, a, pitch, t * NG, tile_cols(t), warp, lane);
  long long t_prev = -1;
  for (int k = 0; t < ntiles; ++k, t_prev = t, t += gridDim.x) {
    const uint32_t buf = (uint32_t)(k & 1) * (H * NG);
    // (a) operands of tile t, per-column eigenvalue parts
    store_tile<H>(regs, bt, warp, lane);
    if (tid < NGC) s_lc[tid] = regs.lc;
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (*s_abort) break;
    // (b) forward products of tile t
    if (tid == 0) {
      issue_products<H, true>(sa, sb, tmem + buf);
      tc::mma_commit(&bar[1]);
    }
    __syncwarp();
    // (c) results of the previous tile, (d) loads of the next one
    if (t_prev >= 0)
      store_result<H>(a.spec, pitch, t_prev * NG, tile_cols(t_prev), t_lane + (buf ^ (H * NG)), lq, ch, lane);
    const long long t_next = t + gridDim.x;
    if (t_next < ntiles) load_tile<H>(regs, a, pitch, t_next * NG, tile_cols(t_next), warp, lane);
    // (e) wait for the forward products, (f) divide by the symbol into the inverse operands
    if (!tc::mbar_wait(&bar[1], k & 1)) {
      *s_abort = 1;
      atomicOr(a.status, 4);
    }
    tc::fence_after_sync();
    {
      const int p = 32 * lq + lane;
#pragma unroll
      for (int h = 0; h < H; ++h) {
        float v[32];
        tc::tmem_ld32(t_lane + buf + h * NG, v);
        const float lz = s_lz[H == 2 ? 2 * p + h : p];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float zq[8];
#pragma unroll
          for (int e = 0; e < 4; ++e) {   // complex column 16 ch + 4 q + e: (re, im)
            const float Lv = lz + s_lc[16 * ch + 4 * q + e];
            float r;
            if (a.mode == 0) r = __fdividef(1.0f, (Lv - a.s_eta2) * Lv + a.c0);
            else r = (Lv == 0.0f) ? 0.0f : __fdividef(1.0f, Lv);
            zq[2 * e] = v[8 * q + 2 * e] * r;
            zq[2 * e + 1] = v[8 * q + 2 * e + 1] * r;
          }
          uint4 hi, lo;
          split8(zq, hi, lo);
          const int o = b_off(p, 32 * ch + 8 * q);
          *reinterpret_cast<uint4*>(bt + 2 * h * kTcOpB + o) = hi;
          *reinterpret_cast<uint4*>(bt + (2 * h + 1) * kTcOpB + o) = lo;
        }
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (*s_abort) break;
    // (g) inverse products of tile t (same accumulators), (h) wait for them
    if (tid == 0) {
      issue_products<H, false>(sa, sb, tmem + buf);
      tc::mma_commit(&bar[2]);
    }
    __syncwarp();
    if (!tc::mbar_wait(&bar[2], k & 1)) {
      *s_abort = 1;
      atomicOr(a.status, 4);
    }
    tc::fence_after_sync();
  }
  // results of the last tile
  if (!*s_abort && t_prev >= 0) {
    const int kl = (int)((t_prev - blockIdx.x) / gridDim.x);
    const uint32_t buf = (uint32_t)(kl & 1) * (H * NG);
    store_result<H>(a.spec, pitch, t_prev * NG, tile_cols(t_prev), t_lane + buf, lq, ch, lane);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * H * NG);
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
  e = cudaFuncSetAttribute(k3_zsolve_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<1>::BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k3_zsolve_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcSmem<2>::BYTES);
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
  const long long tiles = (2 * ncols + kTcNG - 1) / kTcNG;
  const int grid = (int)std::min<long long>(tiles, sm_count());
  if (nz == 256) k3_zsolve_tc<2><<<grid, kTcThreads, TcSmem<2>::BYTES, s>>>(a);
  else k3_zsolve_tc<1><<<grid, kTcThreads, TcSmem<1>::BYTES, s>>>(a);
}

}  // namespace ibpf
