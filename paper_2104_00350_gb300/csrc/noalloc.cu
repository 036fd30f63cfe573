// ib_pf_poisson_solve_noalloc: the pressure Poisson solve for callers that cannot
// allocate device memory.  Its spectrum scratch and transform tables live in one
// file-scope device array instead of cudaMalloc'd buffers.
#include <cmath>
#include <mutex>
#include <string>

#include "ibpf_internal.h"

namespace {

// Largest grid: nx, ny powers of two with 8 <= nx, ny <= 1024 and nx * ny <= 2^19.
constexpr int kMaxN = 1024;
constexpr long long kMaxCells = 1LL << 19;
// doubles: spectrum 2 (nx/2 + 1) ny <= 2^19 + 2 * 1024, tables <= 6 * 1024, plus padding
constexpr size_t kScratchDoubles = (1u << 19) + 16384;

// Every GPU that loads the library holds this array (about 4.3 MB) until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Transform tables of the solve, computed on the device (same definitions as the
// context path: eigenvalues of the periodic / zero-gradient second differences and the
// FFT / cosine-transform twiddles).
__global__ void k_noalloc_tables(int nx, int ny, double h, double* lamx, double* lamy,
                                 double2* twx, double2* twy, double2* wd) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const double c = -4.0 / (h * h);
  if (t <= nx / 2) {
    double sn = sinpi((double)t / (double)nx);
    lamx[t] = c * sn * sn;
  }
  if (t < ny) {
    double sn = sinpi((double)t / (2.0 * (double)ny));
    lamy[t] = c * sn * sn;
    double sa, ca;
    sincospi((double)t / (2.0 * (double)ny), &sa, &ca);
    wd[t] = make_double2(ca, -sa);
  }
  if (t < nx / 2) {
    double sa, ca;
    sincospi(2.0 * (double)t / (double)nx, &sa, &ca);
    twx[t] = make_double2(ca, -sa);
  }
  if (t < ny / 2) {
    double sa, ca;
    sincospi(2.0 * (double)t / (double)ny, &sa, &ca);
    twy[t] = make_double2(ca, -sa);
  }
}

size_t align32(size_t n) { return (n + 31) & ~size_t(31); }

ib_pf_status reject(const std::string& msg, ib_pf_status st) {
  ibpf::set_global_error(msg);
  return st;
}

}  // namespace

extern "C" ib_pf_status ib_pf_poisson_solve_noalloc(const double* rhs, double* out, int nx,
                                                    int ny, double h, void* cuda_stream) {
  const auto pow2 = [](int n) { return n > 0 && (n & (n - 1)) == 0; };
  if (!rhs || !out) return reject("poisson_solve_noalloc: null rhs or out", IB_PF_E_ARG);
  if (!pow2(nx) || !pow2(ny) || nx < 8 || ny < 8 || !(h > 0.0) || !std::isfinite(h))
    return reject("poisson_solve_noalloc: nx, ny must be powers of two >= 8 and h > 0", IB_PF_E_ARG);
  if (nx > kMaxN || ny > kMaxN || (long long)nx * ny > kMaxCells)
    return reject("poisson_solve_noalloc: grid " + std::to_string(nx) + "x" + std::to_string(ny) +
                      " exceeds the fixed scratch (nx, ny <= 1024 and nx*ny <= 524288)",
                  IB_PF_E_ARG);
  // an error left by earlier, unrelated work on this thread is reported as such and not
  // blamed on (or cleared by) this call
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return reject(std::string("poisson_solve_noalloc: a CUDA error is pending from earlier work: ") +
                      cudaGetErrorString(e), IB_PF_E_CUDA);
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return reject(std::string("poisson_solve_noalloc: no usable device: ") + cudaGetErrorString(e),
                  IB_PF_E_CUDA);
  double* base = nullptr;
  {
    // first call on a device: look up the device address of the array (host code only
    // sees a stand-in for it)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      e = cudaGetSymbolAddress((void**)&g_scratch_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        return reject(std::string("poisson_solve_noalloc: cudaGetSymbolAddress: ") +
                          cudaGetErrorString(e), IB_PF_E_CUDA);
      }
    }
    base = g_scratch_ptr[dev];
  }
  // carve the array: spectrum, then the tables, each on a 256-byte boundary
  size_t off = 0;
  double2* spec = reinterpret_cast<double2*>(base + off);
  off += align32(2 * (size_t)(nx / 2 + 1) * ny);
  double* lamx = base + off;
  off += align32((size_t)nx / 2 + 1);
  double* lamy = base + off;
  off += align32((size_t)ny);
  double2* twx = reinterpret_cast<double2*>(base + off);
  off += align32((size_t)nx);
  double2* twy = reinterpret_cast<double2*>(base + off);
  off += align32((size_t)ny);
  double2* wd = reinterpret_cast<double2*>(base + off);
  off += align32(2 * (size_t)ny);
  if (off > kScratchDoubles) return reject("poisson_solve_noalloc: scratch layout overflow", IB_PF_E_ARG);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int nt = (nx > ny ? nx : ny);
  k_noalloc_tables<<<(nt + 255) / 256, 256, 0, s>>>(nx, ny, h, lamx, lamy, twx, twy, wd);
  ibpf::spectral_solve_ptrs(nx, ny, rhs, out, 1, 0.0, 0.0, spec, lamx, lamy, twx, twy, wd, s);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return reject(std::string("poisson_solve_noalloc: launch: ") + cudaGetErrorString(e), IB_PF_E_CUDA);
  return IB_PF_OK;
}
