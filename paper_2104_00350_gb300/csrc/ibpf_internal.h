// Internal declarations of the ib_pf CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "ib_pf.h"

namespace ibpf {

constexpr int kNap = 5;            // averaging points per interpolation point (2D)
constexpr int kNap3 = 7;           // the same in 3D: the cell holding the point + 6 neighbours
constexpr int kNsub = 100;         // subgrid points per direction for alpha (Sec. 4.1.1)
constexpr int kNsub3 = 16;         // subgrid points per direction in 3D (16^3 per volume)
constexpr int kMarchDiv = 100;     // normal-march step h/100 (Sec. 4.1.2)
constexpr int kMarchMax = 1000;    // march limit: 10 h
constexpr int kBisect = 60;        // bisection refinements of the intersect point
constexpr double kEps0 = 1.0e-30;  // epsilon_0 of Eq. NormalVectors_part2

// cell map codes (cmap >= 0 is the ghost index)
constexpr int kCellFluid = -1;
constexpr int kCellSolid = -2;

struct Sph {   // sphere centre and radius
  double x, y, z, r;
};

// A union of spheres with a uniform bin grid over the periodic box: bin b lists every
// sphere whose bounding box, grown by one cell, meets the bin (z bins clamped at the ends).
struct SphereSet {
  const Sph* sph = nullptr;
  const int* bstart = nullptr;    // nb[0] nb[1] nb[2] + 1 offsets into blist
  const int* blist = nullptr;
  int nb[3] = {0, 0, 0};
  double bs[3] = {0, 0, 0};       // bin edge lengths
};

struct WallDev {       // wall predicate parameters as the device sees them
  int kind;
  double p0, p1, w;    // w = (2 pi) * p[2]
  double lx = 0, ly = 0, lz = 0;   // 3D: box (periodic images in x and y)
  SphereSet ss;                    // 3D SPHERE / SPHERES
  // MASK: the cell-centre fractions (the instance's alpha_c table) and the grid they live on
  const double* mask = nullptr;
  int mnx = 0, mny = 0, mnz = 0;
  double mh = 0;
};

// geometry tables of one instance (device pointers, FP64 / int)
// tiles per group of the two-level FP64 mass sum (tile_mass in cell_common.cuh)
constexpr int kMassGroup = 256;

struct Tables {
  double* alpha_c = nullptr;   // ny x nx
  double* alpha_u = nullptr;   // ny x nx
  double* alpha_v = nullptr;   // (ny+1) x nx; 3D: nz x ny x nx (y-faces)
  double* alpha_w = nullptr;   // 3D: (nz+1) x ny x nx (z-faces)
  int* solidc = nullptr;       // ny x nx, 1 where the cell centre is solid
  int* cmap = nullptr;         // ny x nx, ghost index / kCellFluid / kCellSolid
  int ng = 0;
  int* gcell = nullptr;        // ng
  double* nrm = nullptr;       // ng x 2
  double* dn = nullptr;        // ng
  double* gamma = nullptr;     // ng
  int* ap1 = nullptr;          // ng x kNap
  double* w1 = nullptr;
  int* ap2 = nullptr;
  double* w2 = nullptr;
  float* w1f = nullptr;        // FP32 copies of w1, w2 (3D FP32 contexts), made after the
  float* w2f = nullptr;        // FP64 precompute
  int nap = kNap;              // averaging points per interpolation point (5 2D, 7 3D)
  int nfu = 0, nfv = 0, nfw = 0;
  int* fu = nullptr;           // nfu linear x1-face indices
  int* fv = nullptr;           // nfv linear x2-face indices
  int* fw = nullptr;           // 3D: nfw linear z-face indices
  int n_fallback = 0;
};

struct Instance {
  int dim = 2;
  int nx = 0, ny = 0, lognx = 0, logny = 0;
  int nz = 1, lognz = 0;       // 3D
  double lx = 0, ly = 0, lz = 0, h = 0;
  ib_pf_geometry geom{};
  ib_pf_params prm{};
  bool prm_ns_semi = false;    // semi-implicit momentum predictor (ns_scheme 1)
  WallDev wall{};
  Tables tab;
  // state, element type of the context; index cur of each pair is level n
  void* C[2] = {nullptr, nullptr};
  void* Clo[2] = {nullptr, nullptr};   // FP32 path: low parts of the compensated C state
  void* U[2] = {nullptr, nullptr};
  void* V[2] = {nullptr, nullptr};
  void* P[2] = {nullptr, nullptr};
  void* Hu = nullptr;
  void* Hv = nullptr;
  void* W[2] = {nullptr, nullptr};   // 3D z-face velocity
  void* Hw = nullptr;
  float* alpha_f = nullptr;          // 3D FP32 form: alpha_u, alpha_v, alpha_w in FP32
  Sph* sph = nullptr;                // 3D sphere set (device copies)
  int* bstart = nullptr;
  int* blist = nullptr;
  // scratch of one step
  void* Q = nullptr;       // CH right-hand side (cells)
  void* phi = nullptr;     // chemical potential (cells)
  void* rhs = nullptr;     // Poisson right-hand side (cells)
  void* phat = nullptr;    // 2P^n - P^{n-1} (cells)
  void* dp = nullptr;      // pressure increment P^{n+1} - P^ (cells)
  void* spec = nullptr;    // ny x (nx/2+1) complex spectrum
  void* gu = nullptr;      // ng ghost-cell velocities
  void* gv = nullptr;
  void* gw = nullptr;      // 3D
  void* fval = nullptr;    // nfu + nfv (+ nfw) re-interpolated face values
  void* ci = nullptr;      // dynamic angle (mu_f > 0): ng wall values C_I (state)
  void* gq = nullptr;      // dynamic angle: ng x (2 + dim) scratch (C_G, B, dC/dx_t)
  // transform tables
  double* lamx = nullptr;  // nx/2+1 eigenvalues of the periodic second difference
  double* lamy = nullptr;  // ny eigenvalues of the Neumann second difference
  float* lamx_f = nullptr; // the same eigenvalues rounded to FP32 (FP32 path symbol)
  float* lamy_f = nullptr;
  void* twx = nullptr;     // nx/2 complex exp(-2 pi i k/nx), element type
  void* twy = nullptr;     // ny/2 complex exp(-2 pi i k/ny)
  void* wdct = nullptr;    // ny complex exp(-i pi m/(2 ny)); 3D: nz entries
  // 3D: lamy holds the ny eigenvalues of the periodic y second difference, twy the ny/2
  // y-FFT twiddles; the wall-normal z axis has its own tables
  // semi-implicit momentum predictor (ns_scheme 1): the wall-normal eigenvalues of the
  // velocity components (FP64 and FP32 copies) and the twiddles of the doubled length
  double* lam_s2 = nullptr;  // DST-II (no-slip ghost rows), in the cosine order k: -(4/h^2) cos^2(pi k/(2n))
  double* lam_d1 = nullptr;  // DST-I (zero wall faces), modes 0..n: -(4/h^2) sin^2(pi m/(2n))
  float* lam_s2_f = nullptr;
  float* lam_d1_f = nullptr;
  void* tw2 = nullptr;       // n complex exp(-2 pi i k/(2n))
  double* lamz = nullptr;  // nz eigenvalues of the Neumann second difference
  float* lamz_f = nullptr;
  void* twz = nullptr;     // nz/2 complex exp(-2 pi i k/nz)
  // reductions
  double* partial = nullptr;   // per-block partial sums
  unsigned* ticket = nullptr;  // last-block counter
  double* mass = nullptr;      // sum of C after the last step
  int* status = nullptr;       // 1 once a non-finite value was seen
  int nblk_red = 0;            // partial sums of the mass reduction (plus their groups)
  // 3D schedule choices (0: the built-in default), set by ib_pf_set_tuning / ib_pf_autotune:
  // row bytes of the y and z transform tiles (64 or 128), planes per predictor block
  int tune_y_rb = 0, tune_z_rb = 0, tune_pred_planes = 0;
  // FP32_3XBF16: the z solve runs on the tensor cores from the split DCT matrices dmat_z
  bool tc_z = false;
  void* dmat_z = nullptr;
  std::vector<void*> bound;    // caller-owned field buffers (ib_pf_bind_fields): never freed
};

// Optional event recorder: mark(name) is called after every kernel launch of a step.
struct Recorder {
  std::vector<cudaEvent_t>* events = nullptr;   // events[0] is recorded before the step
  std::vector<const char*>* names = nullptr;
  size_t next = 0;
  cudaError_t err = cudaSuccess;
  void start(cudaStream_t s) {
    if (!events) return;
    if (events->empty()) {
      cudaEvent_t e;
      if ((err = cudaEventCreate(&e)) != cudaSuccess) return;
      events->push_back(e);
    }
    cudaEventRecordWithFlags((*events)[0], s, cudaEventRecordExternal);
    next = 1;
  }
  void mark(const char* name, cudaStream_t s) {
    if (!events) return;
    if (events->size() <= next) {
      cudaEvent_t e;
      if ((err = cudaEventCreate(&e)) != cudaSuccess) return;
      events->push_back(e);
    }
    if (names->size() < next) names->resize(next, nullptr);
    (*names)[next - 1] = name;
    cudaEventRecordWithFlags((*events)[next], s, cudaEventRecordExternal);
    ++next;
  }
};

struct Ctx {
  int dim = 2;
  int ch_scheme = IB_PF_CH_SEMI_IMPLICIT;
  bool dynamic = false;    // some instance has a dynamic contact angle (mu_f > 0)
  int ns_scheme = IB_PF_NS_EXPLICIT;   // momentum predictor, shared by all instances
  std::vector<Instance> inst;
  int precision = IB_PF_FP64;
  size_t esz = 8;
  cudaStream_t user_stream = nullptr;
  cudaStream_t work = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool geometry_ready = false;
  bool weights_ready = false;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int cur = 0;
  long long steps = 0;
  int launches_per_step = 0;
  int* h_status = nullptr;   // pinned copy of the status words
  void* plan = nullptr;      // BatchPlan of the batched launches (batch.h)
  bool timing = false;
  std::vector<cudaEvent_t> tev;        // timing events of the step graphs
  std::vector<const char*> tnames;     // kernel name of interval k (between tev[k], tev[k+1])
  std::string err;
};

// ---- geometry.cu
cudaError_t geometry_init(Instance& in, cudaStream_t s, std::string& err);
cudaError_t geometry_weights(Instance& in, cudaStream_t s, int* n_fail, std::string& err);

// Epilogue of the inverse row transform (see k_rows_inv): kind 0 plain, 1 add the BDF2
// predictor (2a - b/2)/1.5, 2 store the increment in delta and add a.
// With a_lo/b_lo/out_lo set (FP32 path), kind 1 updates the compensated pair (hi, lo)
// of C exactly: C^{n+1} = (a + a_lo) + ((a + a_lo - b - b_lo)/3 + z) with TwoSum.
// kind 3 (semi-implicit momentum predictor): out = alpha (a + z), the penalised u** from
// u^n = a and the increment z (Eq. Penalization2).
struct EpiArgs {
  int kind = 0;
  const void* a = nullptr;
  const void* b = nullptr;
  void* delta = nullptr;
  const void* a_lo = nullptr;
  const void* b_lo = nullptr;
  void* out_lo = nullptr;
  const void* alpha = nullptr;
};

// ---- spectral.cu: solve in the real-Fourier (x1) x cosine (x2) basis.
// mode 0: (L^2 - (S/Cn^2) L + 1.5 Pe/(Cn^2 dt))^{-1};  mode 1: L^{-1} with the mean mode 0.
cudaError_t spectral_tables(Instance& in, int precision);
// the same three FP64 kernels on caller-supplied spectrum and table pointers
int spectral_solve_ptrs(int nx, int ny, const double* rhs, double* out, int mode, double s_eta2,
                        double c0, double2* spec, const double* lamx, const double* lamy,
                        const double2* twx, const double2* twy, const double2* wd,
                        cudaStream_t s);

// ---- ib_pf_api.cu: message returned by ib_pf_last_error(NULL)
void set_global_error(const std::string& msg);

// ---- step2d.cu (batched step: see batch.h)
int mass_reduce(Instance& in, int precision, const void* C, const void* Clo, cudaStream_t s);

// ---- geometry3d.cu: Sec. 4.1 in 3D (alpha, classes, ghosts, faces; weights)
cudaError_t geometry3_init(Instance& in, const double* h_spheres, int n_spheres,
                           cudaStream_t s, std::string& err);
cudaError_t geometry3_weights(Instance& in, cudaStream_t s, int* n_fail, std::string& err);

// ---- spectral.cu / step3d.cu: the 3D step, one instance after another
cudaError_t spectral3_tables(Instance& in, int precision);
// FP32 copies of the averaging weights of a 3D FP32 instance (after its precompute)
cudaError_t weights3_f32(Instance& in, cudaStream_t s);
// mean ms per launch of the 3D predictor with `planes` planes per block (AB2 history saved
// and restored); -1 on a CUDA error
float step3d_time_predict(const Ctx& c, Instance& in, int planes, int reps, cudaStream_t s);
// mean ms per launch of the 3D y transforms (axis 1) or z solve (axis 2) with rb-byte tile
// rows, timed on the instance's spectral scratch; -1 when rb is not built for that length
float spectral3_time_tiles(const Instance& in, int precision, int axis, int rb, int reps,
                           cudaStream_t s);
// tensor-core z solve of the FP32_3XBF16 form (tc_zsolve.cu)
bool zsolve_tc_supported(int nz);
cudaError_t zsolve_tc_tables(int nz, void** out);
void zsolve_tc_launch(float* spec, int nz, long long ncols, int sp, int nh1, const float* lamz,
                      const float* lamx, const float* lamyp, const void* dmat, int mode, float s_eta2,
                      float c0, int* status, cudaStream_t s);
int spectral3_solve(const Instance& in, int precision, int mode, int cur, cudaStream_t s,
                    Recorder* rec);
int step3d(const Ctx& c, int cur, cudaStream_t s, Recorder* rec);
cudaError_t step3d_setup(Ctx& c);     // FP32 copies of the face fractions

}  // namespace ibpf
