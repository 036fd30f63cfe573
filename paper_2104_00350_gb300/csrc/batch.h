// Device-side view of a context for the batched step kernels: one descriptor per
// instance and, per kernel family, a table mapping each launched block to
// (instance, block within the instance).  Every sub-step is one launch over all instances.
#pragma once

#include <cuda_runtime.h>

#include "ibpf_internal.h"

namespace ibpf {

template <typename T> struct C2T;
template <> struct C2T<double> { using type = double2; };
template <> struct C2T<float> { using type = float2; };

// kernel families and their work units
enum Family {
  kFamCell = 0,    // 32 x 32 tiles of cells / faces (32 x 8 threads, 4 rows each)
  kFamRows = 1,    // groups of fft_rows_per_block(nx) pairs of x1 rows (row FFTs)
  kFamCols = 2,    // groups of fft_cols_per_block(ny) spectral columns (x2 transforms + symbol)
  kFamGhost = 3,   // chunks of kGhostChunk ghosts
  kFamFace = 4,    // chunks of kGhostChunk re-interpolated faces
  kFamRowsL = 5,   // as kFamRows for rows of 2048 or 4096 points
  kFamColsL = 6,   // as kFamCols for columns of 2048 points
  kFamD1 = 7,      // semi-implicit predictor: groups of DST-I columns (2 ny-point FFTs)
  kFamD1L = 8,     // the same for 2 ny of 2048 or 4096 points
  kNumFam = 9
};
constexpr int kTileX = 32, kTileY = 8;       // threads of a cell-family block
constexpr int kRowsPerThread = 4;            // cells per thread along x2
constexpr int kTileH = kTileY * kRowsPerThread;   // cell tile: 32 x 32
// Transform blocks hold 8 complex points per thread in registers during a pass: 128 threads
// (1024 points: several transforms of up to 1024 points) or, for 2048 and 4096 points, 512
// threads (4096 points).  Each class is its own launch.
constexpr int kFftSmallThreads = 128;
constexpr int kFftLargeThreads = 512;
__host__ __device__ constexpr int fft_threads(int n) {
  return n <= 8 * kFftSmallThreads ? kFftSmallThreads : kFftLargeThreads;
}
__host__ __device__ constexpr int fft_per_block(int n) { return 8 * fft_threads(n) / n; }
// shared-memory slots of a transform buffer of e points: one pad slot per 16 points
__host__ __device__ constexpr int fft_buf(int e) { return e + (e >> 4); }
// row pitch of the 3D half spectrum: nx/2 + 1 rounded up to even (16-byte aligned rows)
__host__ __device__ constexpr int spec3_pitch(int nx) { return (nx / 2 + 2) & ~1; }
// dynamic shared memory of a column-transform block of eb points for columns of n points:
// points, twiddles and cosine weights (complex) and two eigenvalue parts per column.  nmin:
// the shortest column length the block may get (most columns per block) when one size
// serves several lengths up to n.
template <typename T>
constexpr size_t cols_smem_bytes(int n, int eb, int nmin = 0) {
  return sizeof(typename C2T<T>::type) * (size_t)(fft_buf(eb) + n / 2 + n) +
         sizeof(T) * (size_t)(2 * (eb / (nmin ? nmin : n)));
}
constexpr int kGhostChunk = 128;

template <typename T>
struct StepArgs {
  int nx, ny;
  T inv_h, inv_h2, dt;
  // Cahn-Hilliard
  T S, inv_eta2, pe_eta2, inv_dt, eta2;
  T inv_pe;   // 1/Pe (explicit variant)
  // fluid properties: rho(C) = rho_a + rho_b C, mu(C) = mu_a + mu_b C
  T rho_a, rho_b, mu_a, mu_b, rho0, inv_rho0, Re, k_st;
  // contact angle / slip
  double k_wet;   // kappa Cn
  double cos_th;
  double l_s;
  // dynamic angle (mu_f > 0): a_dyn = dt / (mu_f Cn), 0 for the static angle
  double a_dyn;
  double inv_ca;  // 1 / Ca
  double mf_coef; // semi-implicit predictor: (rho_l - rho_g) / (2 Pe)
};

template <typename T>
struct InstDev {
  using C2 = typename C2T<T>::type;
  int nx, ny, lognx, logny, gx;   // gx: tiles along x1
  StepArgs<T> a;
  T* C[2];
  T* Clo[2];
  T* U[2];
  T* V[2];
  T* P[2];
  T* Hu;
  T* Hv;
  T* Q;
  T* phi;
  T* rhs;
  T* phat;
  T* dp;
  C2* spec;
  T* gu;
  T* gv;
  T* fval;
  double* ci;  // dynamic angle: per-ghost wall value C_I (state, FP64 in both forms)
  T* gq;       // dynamic angle: per-ghost scratch C_G, B, (dC/dx_t)_I
  Tables tab;
  const T* au;                // face fractions alpha_u, alpha_v in the field type
  const T* av;
  const double* lamx;
  const double* lamy;
  const float* lamx_f;
  const float* lamy_f;
  const C2* twx;
  const C2* twy;
  const C2* wd;
  double s_eta2, c0;          // CH symbol: L^2 - s_eta2 L + c0
  double a_visc;              // semi-implicit predictor: (1 - a_visc L), a_visc = dt nu0 / 2
  const double* lam_s2;       // its wall-normal eigenvalues (DST-II, cosine order; DST-I)
  const double* lam_d1;
  const float* lam_s2_f;
  const float* lam_d1_f;
  const C2* tw2;              // twiddles of the 2 ny-point FFTs
  double* partial;
  unsigned* ticket;
  double* mass;
  int* status;
};

// host-side bookkeeping of the batched launches (owned by the context)
struct BatchPlan {
  void* d_inst = nullptr;              // InstDev<T>[n]
  void* alpha_f = nullptr;             // FP32 form: FP32 copies of alpha_u, alpha_v
  int2* d_blk[kNumFam] = {};           // (instance, local block) per launched block
  int nblk[kNumFam] = {};
  size_t rows_smem[2] = {}, cols_smem[2] = {};   // small / large transform class
  size_t d1_smem[2] = {};                          // DST-I blocks
  int max_nx = 0, max_ny = 0;
};

cudaError_t batch_setup(Ctx& c, BatchPlan& plan);
void batch_free(BatchPlan& plan);
int step_batch(const Ctx& c, const BatchPlan& plan, int cur, cudaStream_t s, Recorder* rec);

// batched spectral kernels (spectral.cu); src selects Q (0) or rhs (1)
template <typename T>
int spectral_solve_batch(const BatchPlan& plan, int mode, int cur, cudaStream_t s,
                         Recorder* rec);

}  // namespace ibpf
