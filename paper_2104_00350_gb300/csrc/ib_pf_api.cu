// C ABI of the ib_pf library: context life cycle, field I/O and step replay through CUDA
// graphs.  Declarations and argument contracts are in include/ib_pf.h.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <algorithm>

#include "batch.h"
#include "ibpf_internal.h"

using namespace ibpf;

namespace {

std::string g_create_error;

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      ctx->err = std::string(#call) + " failed: " + cudaGetErrorString(e_);       \
      return IB_PF_E_CUDA;                                                        \
    }                                                                             \
  } while (0)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

ib_pf_status fail(ib_pf_ctx* c, ib_pf_status st, const std::string& msg);

size_t field_elems(const Instance& in, int id) {
  const size_t nxy = (size_t)in.nx * in.ny, cells = nxy * in.nz;
  switch (id) {
    case IB_PF_F_V: case IB_PF_F_V_OLD: case IB_PF_F_HV:
      return in.dim == 3 ? cells : cells + in.nx;
    case IB_PF_F_W: case IB_PF_F_W_OLD: case IB_PF_F_HW: return cells + nxy;
    case IB_PF_F_C_I: return (size_t)in.tab.ng;
    default: return cells;
  }
}

void* field_ptr(Ctx& c, Instance& in, int id) {
  const int n = c.cur, o = 1 - c.cur;
  switch (id) {
    case IB_PF_F_C: return in.C[n];
    case IB_PF_F_C_OLD: return in.C[o];
    case IB_PF_F_U: return in.U[n];
    case IB_PF_F_U_OLD: return in.U[o];
    case IB_PF_F_V: return in.V[n];
    case IB_PF_F_V_OLD: return in.V[o];
    case IB_PF_F_HU: return in.Hu;
    case IB_PF_F_HV: return in.Hv;
    case IB_PF_F_P: return in.P[n];
    case IB_PF_F_P_OLD: return in.P[o];
    case IB_PF_F_PHI: return in.phi;
    case IB_PF_F_Q: return in.Q;
    case IB_PF_F_RHS_P: return in.rhs;
    case IB_PF_F_C_LO: return in.Clo[n];
    case IB_PF_F_C_OLD_LO: return in.Clo[o];
    case IB_PF_F_W: return in.W[n];
    case IB_PF_F_W_OLD: return in.W[o];
    case IB_PF_F_HW: return in.Hw;
    case IB_PF_F_C_I: return in.ci;
    default: return nullptr;
  }
}

void free_instance(Instance& in) {
  void* ptrs[] = {in.C[0], in.C[1], in.Clo[0], in.Clo[1], in.U[0], in.U[1], in.V[0], in.V[1], in.P[0], in.P[1],
                  in.Hu, in.Hv, in.Q, in.phi, in.rhs, in.phat, in.dp, in.spec, in.gu, in.gv, in.fval,
                  in.lamx, in.lamy, in.lamx_f, in.lamy_f, in.twx, in.twy, in.wdct, in.partial, in.ticket, in.mass,
                  in.status, in.tab.alpha_c, in.tab.alpha_u, in.tab.alpha_v, in.tab.solidc,
                  in.tab.cmap, in.tab.gcell, in.tab.nrm, in.tab.dn, in.tab.gamma, in.tab.ap1,
                  in.tab.w1, in.tab.ap2, in.tab.w2, in.tab.fu, in.tab.fv, in.W[0], in.W[1], in.Hw,
                  in.gw, in.lamz, in.lamz_f, in.twz, in.sph, in.bstart, in.blist,
                  in.tab.alpha_w, in.tab.fw, in.alpha_f, in.ci, in.gq, in.lam_s2, in.lam_d1,
                  in.lam_s2_f, in.lam_d1_f, in.tw2, in.tab.w1f, in.tab.w2f, in.dmat_z};
  for (void* p : ptrs) {
    if (!p) continue;
    bool caller_owned = false;
    for (void* b : in.bound) caller_owned = caller_owned || b == p;
    if (!caller_owned) cudaFree(p);
  }
}

// order the work stream after everything already queued on the caller's stream
cudaError_t join_in(Ctx& c) {
  if (c.work == c.user_stream) return cudaSuccess;
  cudaError_t e = cudaEventRecord(c.ev_in, c.user_stream);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(c.work, c.ev_in, 0);
}

// order the caller's stream after everything queued on the work stream
cudaError_t join_out(Ctx& c) {
  if (c.work == c.user_stream) return cudaSuccess;
  cudaError_t e = cudaEventRecord(c.ev_out, c.work);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(c.user_stream, c.ev_out, 0);
}

}  // namespace

struct ib_pf_ctx : public Ctx {};

namespace ibpf {
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace ibpf

namespace {
ib_pf_status fail(ib_pf_ctx* c, ib_pf_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return st;
}

// a MASK geometry's volume fractions: present, finite, in [0, 1]
bool mask_ok(const double* a, size_t n, std::string& why) {
  if (!a) {
    why = "MASK needs the volume fractions (ib_pf_geometry.alpha)";
    return false;
  }
  for (size_t i = 0; i < n; ++i)
    if (!(a[i] >= 0.0 && a[i] <= 1.0)) {
      why = "MASK volume fraction " + std::to_string(i) + " is not in [0, 1]";
      return false;
    }
  return true;
}

ib_pf_status validate3(const ib_pf_grid& g, const ib_pf_geometry& w, std::string& why) {
  for (int a = 0; a < 3; ++a) {
    if (!is_pow2(g.n[a]) || g.n[a] < 8 || g.n[a] > 1024) {
      why = "3D: nx, ny, nz must be powers of two with 8 <= n <= 1024";
      return IB_PF_E_ARG;
    }
    if (!(g.L[a] > 0)) { why = "domain lengths must be positive"; return IB_PF_E_ARG; }
  }
  const double hx = g.L[0] / g.n[0];
  if (std::fabs(g.L[1] / g.n[1] - hx) > 1e-12 * hx || std::fabs(g.L[2] / g.n[2] - hx) > 1e-12 * hx) {
    why = "cells must be cubes (lx/nx == ly/ny == lz/nz)";
    return IB_PF_E_ARG;
  }
  if (w.kind != IB_PF_WALL_FLAT && w.kind != IB_PF_WALL_SPHERE && w.kind != IB_PF_WALL_SPHERES &&
      w.kind != IB_PF_WALL_NONE && w.kind != IB_PF_WALL_MASK) {
    why = "3D wall kind must be FLAT, SPHERE, SPHERES, MASK or NONE";
    return IB_PF_E_ARG;
  }
  if (w.kind == IB_PF_WALL_MASK) {
    const size_t nc = (size_t)g.n[0] * g.n[1] * g.n[2];
    if (!mask_ok(w.alpha, 4 * nc + (size_t)g.n[0] * g.n[1], why)) return IB_PF_E_ARG;
  }
  if (w.kind == IB_PF_WALL_SPHERE && !(w.p[3] > 0)) { why = "sphere radius must be positive"; return IB_PF_E_ARG; }
  if (w.kind == IB_PF_WALL_SPHERES) {
    if (!w.spheres || w.n_spheres < 1) { why = "SPHERES needs a sphere array"; return IB_PF_E_ARG; }
    for (int q = 0; q < w.n_spheres; ++q)
      if (!(w.spheres[4 * q + 3] > 0) || !std::isfinite(w.spheres[4 * q]) ||
          !std::isfinite(w.spheres[4 * q + 1]) || !std::isfinite(w.spheres[4 * q + 2])) {
        why = "sphere " + std::to_string(q) + ": finite centre and positive radius required";
        return IB_PF_E_ARG;
      }
  }
  return IB_PF_OK;
}

ib_pf_status validate(const ib_pf_grid& g, const ib_pf_geometry& w, const ib_pf_params& p,
                      std::string& why) {
  if (g.dim != 2 && g.dim != 3) { why = "dim must be 2 or 3"; return IB_PF_E_ARG; }
  if (p.ch_scheme != IB_PF_CH_SEMI_IMPLICIT && p.ch_scheme != IB_PF_CH_EXPLICIT) {
    why = "unknown ch_scheme";
    return IB_PF_E_ARG;
  }
  if (p.weights != IB_PF_W_LINEAR && p.weights != IB_PF_W_IDW) {
    why = "unknown weights";
    return IB_PF_E_ARG;
  }
  if (p.ns_scheme != IB_PF_NS_EXPLICIT && p.ns_scheme != IB_PF_NS_SEMI_IMPLICIT) {
    why = "unknown ns_scheme";
    return IB_PF_E_ARG;
  }
  if (p.ns_scheme == IB_PF_NS_SEMI_IMPLICIT && g.dim == 3) {
    why = "the semi-implicit momentum predictor is built for 2D contexts";
    return IB_PF_E_UNSUPPORTED;
  }
  if (g.dim == 3) {
    if (p.precision != IB_PF_FP64 && p.precision != IB_PF_FP32 && p.precision != IB_PF_FP32_3XBF16) {
      why = "unknown precision";
      return IB_PF_E_ARG;
    }
    if (p.precision == IB_PF_FP32_3XBF16 && !zsolve_tc_supported(g.n[2])) {
      why = "the tensor-core z solve (FP32_3XBF16) is built for nz = 128 and 256";
      return IB_PF_E_UNSUPPORTED;
    }
    if (!(p.mu_f >= 0.0) || !std::isfinite(p.mu_f)) { why = "mu_f must be finite and >= 0"; return IB_PF_E_ARG; }
    const double vals3[] = {p.Re, p.Ca, p.Cn, p.Pe, p.rho_ratio, p.mu_ratio, p.dt, p.d1, p.d2};
    for (double v : vals3)
      if (!(v > 0) || !std::isfinite(v)) { why = "Re, Ca, Cn, Pe, ratios, dt, d1, d2 must be positive"; return IB_PF_E_ARG; }
    if (!(p.S >= 0) || !(p.l_s >= 0) || !std::isfinite(p.theta_deg)) { why = "S, l_s must be >= 0"; return IB_PF_E_ARG; }
    ib_pf_status st = validate3(g, w, why);
    if (st != IB_PF_OK) return st;
    if (!(p.d2 < p.d1) || !(p.d1 > 0.5 * std::sqrt(3.0) * (g.L[0] / g.n[0]))) {
      why = "need d1 > half the cell diagonal and d2 < d1 (Sec. 4.1.2)";
      return IB_PF_E_ARG;
    }
    return IB_PF_OK;
  }
  const int nx = g.n[0], ny = g.n[1];
  if (!is_pow2(nx) || !is_pow2(ny) || nx < 8 || ny < 8 || nx > 4096 || ny > 2048) {
    why = "nx, ny must be powers of two with 8 <= nx <= 4096 and 8 <= ny <= 2048";
    return IB_PF_E_ARG;
  }
  if (!(g.L[0] > 0) || !(g.L[1] > 0)) { why = "domain lengths must be positive"; return IB_PF_E_ARG; }
  const double hx = g.L[0] / nx, hy = g.L[1] / ny;
  if (std::fabs(hx - hy) > 1e-12 * hx) { why = "cells must be square (lx/nx == ly/ny)"; return IB_PF_E_ARG; }
  if (w.kind != IB_PF_WALL_FLAT && w.kind != IB_PF_WALL_SINUSOID && w.kind != IB_PF_WALL_NONE &&
      w.kind != IB_PF_WALL_MASK) {
    why = "unknown wall kind";
    return IB_PF_E_ARG;
  }
  if (w.kind == IB_PF_WALL_MASK && !mask_ok(w.alpha, (size_t)(3 * ny + 1) * nx, why)) return IB_PF_E_ARG;
  if (p.precision == IB_PF_FP32_3XBF16) {
    why = "FP32_3XBF16 (tensor-core z solve) is built for 3D contexts";
    return IB_PF_E_UNSUPPORTED;
  }
  if (p.precision != IB_PF_FP64 && p.precision != IB_PF_FP32) { why = "unknown precision"; return IB_PF_E_ARG; }
  if (!(p.mu_f >= 0.0) || !std::isfinite(p.mu_f)) { why = "mu_f must be finite and >= 0"; return IB_PF_E_ARG; }
  const double vals[] = {p.Re, p.Ca, p.Cn, p.Pe, p.rho_ratio, p.mu_ratio, p.dt, p.d1, p.d2};
  for (double v : vals)
    if (!(v > 0) || !std::isfinite(v)) { why = "Re, Ca, Cn, Pe, ratios, dt, d1, d2 must be positive"; return IB_PF_E_ARG; }
  if (!(p.S >= 0) || !(p.l_s >= 0) || !std::isfinite(p.theta_deg)) { why = "S, l_s must be >= 0"; return IB_PF_E_ARG; }
  if (!(p.d2 < p.d1) || !(p.d1 > 0.5 * std::sqrt(2.0) * hx)) {
    why = "need d1 > half the cell diagonal and d2 < d1 (Sec. 4.1.2)";
    return IB_PF_E_ARG;
  }
  return IB_PF_OK;
}

ib_pf_status capture_graphs(ib_pf_ctx* ctx) {
  for (int ph = 0; ph < 2; ++ph) {
    if (ctx->graph[ph]) continue;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->work, cudaStreamCaptureModeThreadLocal));
    int launches = 0;
    Recorder rec;
    if (ctx->timing) {
      rec.events = &ctx->tev;
      rec.names = &ctx->tnames;
      rec.start(ctx->work);
    }
    launches = ctx->dim == 3
                   ? step3d(*ctx, ph, ctx->work, ctx->timing ? &rec : nullptr)
                   : step_batch(*ctx, *(BatchPlan*)ctx->plan, ph, ctx->work, ctx->timing ? &rec : nullptr);
    for (size_t k = 0; k < ctx->inst.size(); ++k) {
      cudaMemcpyAsync(ctx->h_status + k, ctx->inst[k].status, sizeof(int), cudaMemcpyDeviceToHost,
                      ctx->work);
    }
    cudaError_t e = cudaStreamEndCapture(ctx->work, &g);
    if (e != cudaSuccess) return fail(ctx, IB_PF_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    if (rec.err != cudaSuccess) {
      cudaGraphDestroy(g);
      return fail(ctx, IB_PF_E_CUDA, std::string("timing events: ") + cudaGetErrorString(rec.err));
    }
    e = cudaGraphInstantiate(&ctx->graph[ph], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ctx, IB_PF_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    ctx->launches_per_step = launches;
  }
  return IB_PF_OK;
}

}  // namespace

extern "C" {

ib_pf_status ib_pf_init_geometry(ib_pf_ctx** out, int n_instances, const ib_pf_grid* grids,
                                 const ib_pf_geometry* geoms, const ib_pf_params* params,
                                 void* cuda_stream) {
  if (!out || n_instances < 1 || !grids || !geoms || !params)
    return fail(nullptr, IB_PF_E_ARG, "null pointer or n_instances < 1");
  *out = nullptr;
  for (int k = 0; k < n_instances; ++k) {
    std::string why;
    ib_pf_status st = validate(grids[k], geoms[k], params[k], why);
    if (st != IB_PF_OK) return fail(nullptr, st, "instance " + std::to_string(k) + ": " + why);
    if (params[k].precision != params[0].precision)
      return fail(nullptr, IB_PF_E_ARG, "all instances must share one precision");
    if (grids[k].dim != grids[0].dim)
      return fail(nullptr, IB_PF_E_ARG, "all instances must share one dimension");
    if (params[k].ch_scheme != params[0].ch_scheme)
      return fail(nullptr, IB_PF_E_ARG, "all instances must share one ch_scheme");
    if (params[k].ns_scheme != params[0].ns_scheme)
      return fail(nullptr, IB_PF_E_ARG, "all instances must share one ns_scheme");
  }
  ib_pf_ctx* ctx = new (std::nothrow) ib_pf_ctx();
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "out of host memory");
  // the split-BF16 form is the FP32 form with the tensor-core z solve (Instance::tc_z)
  ctx->precision = params[0].precision == IB_PF_FP32_3XBF16 ? IB_PF_FP32 : params[0].precision;
  ctx->dim = grids[0].dim;
  ctx->ch_scheme = params[0].ch_scheme;
  ctx->ns_scheme = params[0].ns_scheme;
  ctx->esz = ctx->precision == IB_PF_FP64 ? 8 : 4;
  ctx->user_stream = (cudaStream_t)cuda_stream;
  auto bail = [&](ib_pf_status st) {
    g_create_error = ctx->err;
    ib_pf_destroy(ctx);
    return st;
  };
  if (cudaStreamCreateWithFlags(&ctx->work, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_status, sizeof(int) * n_instances) != cudaSuccess) {
    ctx->err = "CUDA initialisation failed (stream/event/pinned allocation)";
    return bail(IB_PF_E_CUDA);
  }
  std::memset(ctx->h_status, 0, sizeof(int) * n_instances);
  if (join_in(*ctx) != cudaSuccess) { ctx->err = "stream join failed"; return bail(IB_PF_E_CUDA); }
  ctx->inst.resize(n_instances);
  for (int k = 0; k < n_instances; ++k) {
    Instance& in = ctx->inst[k];
    in.dim = grids[k].dim;
    in.nx = grids[k].n[0];
    in.ny = grids[k].n[1];
    in.lognx = ilog2(in.nx);
    in.logny = ilog2(in.ny);
    in.lx = grids[k].L[0];
    in.ly = grids[k].L[1];
    if (in.dim == 3) {
      in.nz = grids[k].n[2];
      in.lognz = ilog2(in.nz);
      in.lz = grids[k].L[2];
    }
    in.h = in.lx / in.nx;
    in.geom = geoms[k];
    in.prm = params[k];
    in.tc_z = params[k].precision == IB_PF_FP32_3XBF16;
    in.prm.precision = ctx->precision;
    in.prm_ns_semi = params[k].ns_scheme == IB_PF_NS_SEMI_IMPLICIT;
    in.wall.kind = geoms[k].kind;
    in.wall.p0 = geoms[k].p[0];
    in.wall.p1 = geoms[k].p[1];
    in.wall.w = (2.0 * M_PI) * geoms[k].p[2];
    const size_t nxy = (size_t)in.nx * in.ny, cells = nxy * in.nz, es = ctx->esz;
    const size_t vf = in.dim == 3 ? cells : cells + in.nx;
    const size_t nh1 = (size_t)in.nx / 2 + 1;
    void** cell_fields[] = {&in.C[0], &in.C[1], &in.P[0], &in.P[1], &in.U[0], &in.U[1], &in.Hu,
                            &in.Q, &in.phi, &in.rhs, &in.phat, &in.dp};
    for (void** f : cell_fields) {
      if (cudaMalloc(f, cells * es) != cudaSuccess) { ctx->err = "field allocation failed"; return bail(IB_PF_E_CUDA); }
      cudaMemsetAsync(*f, 0, cells * es, ctx->work);
    }
    if (ctx->precision == IB_PF_FP32) {
      for (void** f : {&in.Clo[0], &in.Clo[1]}) {
        if (cudaMalloc(f, cells * es) != cudaSuccess) { ctx->err = "field allocation failed"; return bail(IB_PF_E_CUDA); }
        cudaMemsetAsync(*f, 0, cells * es, ctx->work);
      }
    }
    void** vfields[] = {&in.V[0], &in.V[1], &in.Hv};
    for (void** f : vfields) {
      if (cudaMalloc(f, vf * es) != cudaSuccess) { ctx->err = "field allocation failed"; return bail(IB_PF_E_CUDA); }
      cudaMemsetAsync(*f, 0, vf * es, ctx->work);
    }
    if (in.dim == 3) {
      void** wfields[] = {&in.W[0], &in.W[1], &in.Hw};
      for (void** f : wfields) {
        if (cudaMalloc(f, (cells + nxy) * es) != cudaSuccess) { ctx->err = "field allocation failed"; return bail(IB_PF_E_CUDA); }
        cudaMemsetAsync(*f, 0, (cells + nxy) * es, ctx->work);
      }
    }
    // 3D: rows of spec3_pitch(nx) points, the pad column zero for good
    const size_t spec_bytes =
        (size_t)in.ny * in.nz * (in.dim == 3 ? spec3_pitch(in.nx) : nh1) * 2 * es;
    if (cudaMalloc(&in.spec, spec_bytes) != cudaSuccess) {
      ctx->err = "spectral workspace allocation failed";
      return bail(IB_PF_E_CUDA);
    }
    cudaMemsetAsync(in.spec, 0, spec_bytes, ctx->work);
    // partial sums: one per cell tile of the step's reduction, or per 256-cell block of
    // the stand-alone reduction, whichever is more
    const int ntile = ((in.nx + kTileX - 1) / kTileX) * ((in.ny + kTileH - 1) / kTileH);
    // (3D FP32: one partial per warp of the correction kernel, 128 cells)
    const int nred = (int)((cells + (in.dim == 3 ? 127 : 255)) / (in.dim == 3 ? 128 : 256));
    const int nblk = ntile > nred ? ntile : nred;
    in.nblk_red = nblk;
    // group sums and group counters of the two-level final sum (tile_mass)
    const int ngrp = (nblk + kMassGroup - 1) / kMassGroup;
    if (cudaMalloc((void**)&in.partial, sizeof(double) * (nblk + ngrp)) != cudaSuccess ||
        cudaMalloc((void**)&in.ticket, sizeof(unsigned) * (1 + ngrp)) != cudaSuccess ||
        cudaMalloc((void**)&in.mass, sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&in.status, sizeof(int)) != cudaSuccess) {
      ctx->err = "reduction buffers allocation failed";
      return bail(IB_PF_E_CUDA);
    }
    cudaMemsetAsync(in.ticket, 0, sizeof(unsigned) * (1 + ngrp), ctx->work);
    cudaMemsetAsync(in.mass, 0, sizeof(double), ctx->work);
    cudaMemsetAsync(in.status, 0, sizeof(int), ctx->work);
    if ((in.dim == 3 ? spectral3_tables(in, ctx->precision) : spectral_tables(in, ctx->precision)) !=
        cudaSuccess) {
      ctx->err = std::string("transform tables: ") + cudaGetErrorString(cudaGetLastError());
      return bail(IB_PF_E_CUDA);
    }
    std::string gerr;
    const cudaError_t ge = in.dim == 3 ? geometry3_init(in, geoms[k].spheres, geoms[k].n_spheres, ctx->work, gerr)
                                       : geometry_init(in, ctx->work, gerr);
    in.geom.alpha = nullptr;   // the caller's MASK fractions are copied; drop the pointer
    in.geom.spheres = nullptr;
    if (ge != cudaSuccess) {
      ctx->err = "geometry: " + gerr;
      return bail(IB_PF_E_CUDA);
    }
    const Tables& t = in.tab;
    if (cudaMalloc(&in.gu, (size_t)(t.ng ? t.ng : 1) * es) != cudaSuccess ||
        cudaMalloc(&in.gv, (size_t)(t.ng ? t.ng : 1) * es) != cudaSuccess ||
        (in.dim == 3 && cudaMalloc(&in.gw, (size_t)(t.ng ? t.ng : 1) * es) != cudaSuccess) ||
        cudaMalloc(&in.fval, (size_t)(t.nfu + t.nfv + t.nfw + 1) * es) != cudaSuccess) {
      ctx->err = "ghost scratch allocation failed";
      return bail(IB_PF_E_CUDA);
    }
    if (in.prm.mu_f > 0.0) {
      // dynamic angle: wall values C_I (state, unset = NaN) and per-ghost scratch
      const size_t ng1 = (size_t)(t.ng ? t.ng : 1);
      if (cudaMalloc(&in.ci, ng1 * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&in.gq, ng1 * (2 + in.dim) * es) != cudaSuccess) {
        ctx->err = "dynamic-angle scratch allocation failed";
        return bail(IB_PF_E_CUDA);
      }
      cudaMemsetAsync(in.ci, 0xff, ng1 * sizeof(double), ctx->work);
      ctx->dynamic = true;
    }
  }
  if (cudaStreamSynchronize(ctx->work) != cudaSuccess) {
    ctx->err = std::string("init: ") + cudaGetErrorString(cudaGetLastError());
    return bail(IB_PF_E_CUDA);
  }
  if (ctx->dim == 3) {
    cudaError_t e = step3d_setup(*ctx);
    if (e != cudaSuccess) {
      ctx->err = std::string("3D setup: ") + cudaGetErrorString(e);
      return bail(IB_PF_E_CUDA);
    }
  } else {
    BatchPlan* plan = new (std::nothrow) BatchPlan();
    if (!plan) { ctx->err = "out of host memory"; return bail(IB_PF_E_ARG); }
    ctx->plan = plan;
    cudaError_t e = batch_setup(*ctx, *plan);
    if (e != cudaSuccess) {
      ctx->err = std::string("batch plan: ") + cudaGetErrorString(e);
      return bail(IB_PF_E_CUDA);
    }
  }
  join_out(*ctx);
  ctx->geometry_ready = true;
  *out = ctx;
  return IB_PF_OK;
}

ib_pf_status ib_pf_precompute_weights(ib_pf_ctx* ctx) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (!ctx->geometry_ready) return fail(ctx, IB_PF_E_STATE, "geometry not initialised");
  CK(join_in(*ctx));
  int total_fail = 0;
  for (Instance& in : ctx->inst) {
    int nf = 0;
    std::string gerr;
    const cudaError_t ge = in.dim == 3 ? geometry3_weights(in, ctx->work, &nf, gerr)
                                       : geometry_weights(in, ctx->work, &nf, gerr);
    if (ge != cudaSuccess)
      return fail(ctx, IB_PF_E_CUDA, "weights: " + gerr);
    if (in.dim == 3 && ctx->precision == IB_PF_FP32) CK(weights3_f32(in, ctx->work));
    total_fail += nf;
  }
  CK(join_out(*ctx));
  if (total_fail > 0)
    return fail(ctx, IB_PF_E_GEOMETRY, std::to_string(total_fail) + " ghost(s) without an intersect point within 10 h");
  ctx->weights_ready = true;
  return IB_PF_OK;
}

ib_pf_status ib_pf_step(ib_pf_ctx* ctx, int nsteps) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (nsteps < 0) return fail(ctx, IB_PF_E_ARG, "nsteps < 0");
  if (!ctx->weights_ready) return fail(ctx, IB_PF_E_STATE, "ib_pf_precompute_weights has not succeeded");
  for (size_t k = 0; k < ctx->inst.size(); ++k) {
    const int st = ((volatile int*)ctx->h_status)[k];
    if (st & 2)
      return fail(ctx, IB_PF_E_CUDA, "a 3D transform tile failed its alignment check in instance " + std::to_string(k));
    if (st & 4)
      return fail(ctx, IB_PF_E_TIMEOUT, "a tensor-core wait of the z solve gave up in instance " + std::to_string(k));
    if (st != 0)
      return fail(ctx, IB_PF_E_NUMERIC, "non-finite value seen in instance " + std::to_string(k));
  }
  if (nsteps == 0) return IB_PF_OK;
  ib_pf_status st = capture_graphs(ctx);
  if (st != IB_PF_OK) return st;
  CK(join_in(*ctx));
  for (int s = 0; s < nsteps; ++s) {
    CK(cudaGraphLaunch(ctx->graph[ctx->cur], ctx->work));
    ctx->cur = 1 - ctx->cur;
    ++ctx->steps;
  }
  CK(join_out(*ctx));
  return IB_PF_OK;
}

}  // extern "C"

namespace {

// checks of one read (write = false) or write entry; returns the field's device pointer
ib_pf_status check_field(ib_pf_ctx* ctx, int instance, int field_id, const void* buf,
                         long long nbytes, bool write, void** dev) {
  if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, IB_PF_E_ARG, "bad instance");
  if (!buf) return fail(ctx, IB_PF_E_ARG, write ? "null source" : "null destination");
  if (write) {
    const bool lo_field = field_id == IB_PF_F_C_LO || field_id == IB_PF_F_C_OLD_LO;
    const bool w_field = field_id >= IB_PF_F_W && field_id <= IB_PF_F_HW;
    if ((field_id < IB_PF_F_C || field_id > IB_PF_F_P_OLD) && !lo_field && !w_field &&
        field_id != IB_PF_F_C_I)
      return fail(ctx, IB_PF_E_ARG, "field is read-only or unknown");
  }
  Instance& in = ctx->inst[instance];
  void* p = field_ptr(*ctx, in, field_id);
  if (!p) return fail(ctx, IB_PF_E_ARG, "bad field id (low parts of C exist only in FP32 contexts, w only in 3D, "
                          "C_I only with a dynamic contact angle)");
  const size_t es = field_id == IB_PF_F_C_I ? sizeof(double) : ctx->esz;   // C_I is FP64 in both forms
  const long long want = (long long)(field_elems(in, field_id) * es);
  if (nbytes != want) return fail(ctx, IB_PF_E_ARG, "nbytes " + std::to_string(nbytes) + " != " + std::to_string(want));
  *dev = p;
  return IB_PF_OK;
}

// One entry of a batched write, in 32-bit words: dst[i] = src[i] for zhead <= i < words - ztail
// and 0 elsewhere; src == nullptr zeroes all of dst.  src is device memory or the device
// address of pinned (page-locked, mapped) host memory, which the kernel reads directly.
struct CopyEntry {
  const unsigned int* src;
  unsigned int* dst;
  unsigned long long words, zhead, ztail;
  unsigned int fill;   // word written where nothing is copied (0, or all ones: NaN in FP32/FP64)
};
constexpr int kCopyMax = 48;   // 48 entries = 1920 bytes of kernel parameters
struct CopyList {
  CopyEntry e[kCopyMax];
};
constexpr int kCopyThreads = 256, kCopyUnroll = 4;

__global__ void __launch_bounds__(kCopyThreads) k_copy_entries(CopyList L) {
  const CopyEntry c = L.e[blockIdx.y];
  const unsigned long long lo = c.src ? c.zhead : c.words, hi = c.src ? c.words - c.ztail : c.words;
  const unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(c.src) | reinterpret_cast<uintptr_t>(c.dst)) & 15) == 0 &&
                   (c.words & 3) == 0;
  if (vec) {
    // 16-byte words; every vector lies inside [0, words), so a vector that holds any copied
    // word is read whole and its zero words are masked afterwards
    const uint4* s = reinterpret_cast<const uint4*>(c.src);
    uint4* d = reinterpret_cast<uint4*>(c.dst);
    const unsigned long long nv = c.words >> 2;
    for (unsigned long long base = t0; base < nv; base += stride * kCopyUnroll) {
      uint4 v[kCopyUnroll];
#pragma unroll
      for (int u = 0; u < kCopyUnroll; ++u) {   // all loads first: several in flight per thread
        const unsigned long long q = base + u * stride;
        v[u] = make_uint4(c.fill, c.fill, c.fill, c.fill);
        if (q < nv && 4 * q + 4 > lo && 4 * q < hi) v[u] = s[q];
      }
#pragma unroll
      for (int u = 0; u < kCopyUnroll; ++u) {
        const unsigned long long q = base + u * stride;
        if (q >= nv) continue;
        const unsigned long long w0 = 4 * q;
        if (w0 < lo || w0 + 4 > hi) {
          if (w0 + 0 < lo || w0 + 0 >= hi) v[u].x = c.fill;
          if (w0 + 1 < lo || w0 + 1 >= hi) v[u].y = c.fill;
          if (w0 + 2 < lo || w0 + 2 >= hi) v[u].z = c.fill;
          if (w0 + 3 < lo || w0 + 3 >= hi) v[u].w = c.fill;
        }
        d[q] = v[u];
      }
    }
  } else {
    for (unsigned long long i = t0; i < c.words; i += stride)
      c.dst[i] = (i >= lo && i < hi) ? c.src[i] : c.fill;
  }
}

// The effects of a sequence of field writes, gathered so that one launch (per kCopyMax
// entries) performs them: entries keyed by destination, a later write of the same
// destination replacing the earlier one.  Sources that are neither device memory nor
// pinned host memory are copied by cudaMemcpyAsync when added (stream order then puts
// them before the launch, which carries only their zero rows).
struct WritePlan {
  std::vector<CopyEntry> e;
  std::vector<const void*> key;   // destination field of each entry

  void kill(const void* dst) {
    for (size_t q = 0; q < e.size(); ++q)
      if (key[q] == dst) e[q].words = 0;
  }
  void add(const void* field, const CopyEntry& c) {
    e.push_back(c);
    key.push_back(field);
  }
};

// device address of a host or device buffer, or nullptr if a kernel cannot access it
const void* device_source(const void* src, int src_on_host) {
  if (!src_on_host) return src;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, src) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return src;
  return nullptr;
}

// plan one write (already checked): the copy with the zero wall rows / planes of v (2D)
// or w (3D), and the cleared low part of a written C level (FP32 form)
ib_pf_status plan_write(ib_pf_ctx* ctx, WritePlan& plan, int instance, int field_id, void* dst,
                        const void* src, long long nbytes, int src_on_host) {
  Instance& in = ctx->inst[instance];
  const unsigned long long words = (unsigned long long)nbytes / 4;
  unsigned long long zrow = 0;   // words of each zero wall row / plane at both ends
  const bool w_field = field_id >= IB_PF_F_W && field_id <= IB_PF_F_HW;
  if (in.dim == 3 && w_field) zrow = (unsigned long long)in.nx * in.ny * ctx->esz / 4;
  if (in.dim == 2 && (field_id == IB_PF_F_V || field_id == IB_PF_F_V_OLD || field_id == IB_PF_F_HV))
    zrow = (unsigned long long)in.nx * ctx->esz / 4;
  plan.kill(dst);
  const void* dsrc = device_source(src, src_on_host);
  if (dsrc) {
    plan.add(dst, {(const unsigned int*)dsrc, (unsigned int*)dst, words, zrow, zrow});
  } else {
    CK(cudaMemcpyAsync(dst, src, (size_t)nbytes, cudaMemcpyDefault, ctx->work));
    if (zrow) {
      plan.add(dst, {nullptr, (unsigned int*)dst, zrow, 0, 0});
      plan.add(dst, {nullptr, (unsigned int*)dst + (words - zrow), zrow, 0, 0});
    }
  }
  if ((field_id == IB_PF_F_C || field_id == IB_PF_F_C_OLD) && ctx->precision == IB_PF_FP32) {
    void* lo = field_ptr(*ctx, in, field_id == IB_PF_F_C ? IB_PF_F_C_LO : IB_PF_F_C_OLD_LO);
    plan.kill(lo);
    plan.add(lo, {nullptr, (unsigned int*)lo, words, 0, 0});
  }
  if (field_id == IB_PF_F_C && in.ci && in.tab.ng > 0) {
    // a written C^n unsets the wall values C_I of the dynamic angle (all-ones words: NaN);
    // the next step starts them from the new field
    plan.kill(in.ci);
    plan.add(in.ci, {nullptr, (unsigned int*)in.ci, (unsigned long long)in.tab.ng * 2, 0, 0,
                     0xffffffffu});
  }
  return IB_PF_OK;
}

// one k_copy_entries launch per kCopyMax entries on the work stream
ib_pf_status launch_entries(ib_pf_ctx* ctx, const std::vector<CopyEntry>& live) {
  for (size_t a = 0; a < live.size(); a += kCopyMax) {
    CopyList L{};
    const int m = (int)std::min<size_t>(kCopyMax, live.size() - a);
    unsigned long long most = 0;
    for (int q = 0; q < m; ++q) {
      L.e[q] = live[a + q];
      most = std::max(most, L.e[q].words);
    }
    const unsigned long long per_block = 4ull * kCopyThreads * kCopyUnroll;
    const int gx = (int)std::min<unsigned long long>(128, std::max<unsigned long long>(1, (most + per_block - 1) / per_block));
    k_copy_entries<<<dim3(gx, m), kCopyThreads, 0, ctx->work>>>(L);
    CK(cudaGetLastError());
  }
  return IB_PF_OK;
}

// launch the plan's live entries and clear the status words of the written instances
ib_pf_status run_plan(ib_pf_ctx* ctx, WritePlan& plan, const std::vector<char>& touched) {
  for (size_t k = 0; k < touched.size(); ++k)
    if (touched[k]) plan.add(ctx->inst[k].status, {nullptr, (unsigned int*)ctx->inst[k].status, 1, 0, 0});
  std::vector<CopyEntry> live;
  for (const CopyEntry& c : plan.e)
    if (c.words) live.push_back(c);
  return launch_entries(ctx, live);
}

}  // namespace

extern "C" {

ib_pf_status ib_pf_read_fields(ib_pf_ctx* ctx, int instance, int field_id, void* dst,
                               long long nbytes, int dst_on_host) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  void* src = nullptr;
  ib_pf_status st = check_field(ctx, instance, field_id, dst, nbytes, false, &src);
  if (st != IB_PF_OK) return st;
  CK(join_in(*ctx));
  CK(cudaMemcpyAsync(dst, src, (size_t)nbytes, dst_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     ctx->work));
  if (dst_on_host) CK(cudaStreamSynchronize(ctx->work));
  CK(join_out(*ctx));
  return IB_PF_OK;
}

ib_pf_status ib_pf_write_fields(ib_pf_ctx* ctx, int instance, int field_id, const void* src,
                                long long nbytes, int src_on_host) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  void* dst = nullptr;
  ib_pf_status st = check_field(ctx, instance, field_id, src, nbytes, true, &dst);
  if (st != IB_PF_OK) return st;
  CK(join_in(*ctx));
  WritePlan plan;
  st = plan_write(ctx, plan, instance, field_id, dst, src, nbytes, src_on_host);
  if (st != IB_PF_OK) return st;
  std::vector<char> touched(ctx->inst.size(), 0);
  touched[instance] = 1;
  st = run_plan(ctx, plan, touched);
  if (st != IB_PF_OK) return st;
  CK(cudaStreamSynchronize(ctx->work));
  ((volatile int*)ctx->h_status)[instance] = 0;
  CK(join_out(*ctx));
  return IB_PF_OK;
}

ib_pf_status ib_pf_write_fields_batch(ib_pf_ctx* ctx, int n, const int* instances,
                                      const int* field_ids, const void* const* srcs,
                                      const long long* nbytes, int src_on_host) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (n < 0) return fail(ctx, IB_PF_E_ARG, "n < 0");
  if (n == 0) return IB_PF_OK;
  if (!instances || !field_ids || !srcs || !nbytes) return fail(ctx, IB_PF_E_ARG, "null array");
  std::vector<void*> dst(n);
  for (int q = 0; q < n; ++q) {
    ib_pf_status st = check_field(ctx, instances[q], field_ids[q], srcs[q], nbytes[q], true, &dst[q]);
    if (st != IB_PF_OK) return fail(ctx, st, "entry " + std::to_string(q) + ": " + ctx->err);
  }
  CK(join_in(*ctx));
  std::vector<char> touched(ctx->inst.size(), 0);
  WritePlan plan;
  for (int q = 0; q < n; ++q) {
    ib_pf_status st = plan_write(ctx, plan, instances[q], field_ids[q], dst[q], srcs[q], nbytes[q],
                                 src_on_host);
    if (st != IB_PF_OK) return st;
    touched[instances[q]] = 1;
  }
  ib_pf_status rs = run_plan(ctx, plan, touched);
  if (rs != IB_PF_OK) return rs;
  CK(cudaStreamSynchronize(ctx->work));
  for (int q = 0; q < n; ++q) ((volatile int*)ctx->h_status)[instances[q]] = 0;
  CK(join_out(*ctx));
  return IB_PF_OK;
}

ib_pf_status ib_pf_read_fields_batch(ib_pf_ctx* ctx, int n, const int* instances,
                                     const int* field_ids, void* const* dsts,
                                     const long long* nbytes, int dst_on_host) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (n < 0) return fail(ctx, IB_PF_E_ARG, "n < 0");
  if (n == 0) return IB_PF_OK;
  if (!instances || !field_ids || !dsts || !nbytes) return fail(ctx, IB_PF_E_ARG, "null array");
  std::vector<void*> src(n);
  for (int q = 0; q < n; ++q) {
    ib_pf_status st = check_field(ctx, instances[q], field_ids[q], dsts[q], nbytes[q], false, &src[q]);
    if (st != IB_PF_OK) return fail(ctx, st, "entry " + std::to_string(q) + ": " + ctx->err);
  }
  CK(join_in(*ctx));
  // device and pinned host destinations: written by the copy kernel; others: cudaMemcpyAsync
  std::vector<CopyEntry> ent;
  for (int q = 0; q < n; ++q) {
    void* d = const_cast<void*>(device_source(dsts[q], dst_on_host));
    if (d)
      ent.push_back({(const unsigned int*)src[q], (unsigned int*)d, (unsigned long long)nbytes[q] / 4, 0, 0});
    else
      CK(cudaMemcpyAsync(dsts[q], src[q], (size_t)nbytes[q], cudaMemcpyDefault, ctx->work));
  }
  ib_pf_status ls = launch_entries(ctx, ent);
  if (ls != IB_PF_OK) return ls;
  if (dst_on_host) CK(cudaStreamSynchronize(ctx->work));
  CK(join_out(*ctx));
  return IB_PF_OK;
}

ib_pf_status ib_pf_read_table(ib_pf_ctx* ctx, int instance, int table_id, void* dst,
                              long long nbytes, long long* count) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, IB_PF_E_ARG, "bad instance");
  Instance& in = ctx->inst[instance];
  const Tables& t = in.tab;
  const size_t nxy = (size_t)in.nx * in.ny, cells = nxy * in.nz;
  const void* src = nullptr;
  size_t n = 0, es = 8;
  const size_t nap = (size_t)t.nap;
  switch (table_id) {
    case IB_PF_T_ALPHA_C: src = t.alpha_c; n = cells; break;
    case IB_PF_T_ALPHA_U: src = t.alpha_u; n = cells; break;
    case IB_PF_T_ALPHA_V: src = t.alpha_v; n = in.dim == 3 ? cells : cells + in.nx; break;
    case IB_PF_T_CLASS: src = t.cmap; n = cells; es = 4; break;
    case IB_PF_T_GHOST_CELL: src = t.gcell; n = t.ng; es = 4; break;
    case IB_PF_T_NORMAL: src = t.nrm; n = (size_t)in.dim * t.ng; break;
    case IB_PF_T_DN: src = t.dn; n = t.ng; break;
    case IB_PF_T_GAMMA: src = t.gamma; n = t.ng; break;
    case IB_PF_T_AP1: src = t.ap1; n = (size_t)t.ng * nap; es = 4; break;
    case IB_PF_T_W1: src = t.w1; n = (size_t)t.ng * nap; break;
    case IB_PF_T_AP2: src = t.ap2; n = (size_t)t.ng * nap; es = 4; break;
    case IB_PF_T_W2: src = t.w2; n = (size_t)t.ng * nap; break;
    case IB_PF_T_FACE_U: src = t.fu; n = t.nfu; es = 4; break;
    case IB_PF_T_FACE_V: src = t.fv; n = t.nfv; es = 4; break;
    case IB_PF_T_ALPHA_W:
      if (in.dim != 3) return fail(ctx, IB_PF_E_ARG, "alpha_w exists only in 3D");
      src = t.alpha_w; n = cells + nxy; break;
    case IB_PF_T_FACE_W:
      if (in.dim != 3) return fail(ctx, IB_PF_E_ARG, "z-faces exist only in 3D");
      src = t.fw; n = t.nfw; es = 4; break;
    default: return fail(ctx, IB_PF_E_ARG, "bad table id");
  }
  if (table_id >= IB_PF_T_NORMAL && table_id <= IB_PF_T_W2 && !ctx->weights_ready)
    return fail(ctx, IB_PF_E_STATE, "weights not computed");
  if (count) *count = (long long)n;
  if (!dst) return IB_PF_OK;
  if (nbytes != (long long)(n * es)) return fail(ctx, IB_PF_E_ARG, "nbytes does not match the table size");
  CK(join_in(*ctx));
  if (n > 0) CK(cudaMemcpyAsync(dst, src, n * es, cudaMemcpyDeviceToHost, ctx->work));
  CK(cudaStreamSynchronize(ctx->work));
  if (table_id == IB_PF_T_CLASS) {   // cmap -> 0 fluid, 1 ghost, 2 solid
    int* c = (int*)dst;
    for (size_t k = 0; k < n; ++k) c[k] = c[k] >= 0 ? 1 : (c[k] == kCellSolid ? 2 : 0);
  }
  return IB_PF_OK;
}

ib_pf_status ib_pf_query(ib_pf_ctx* ctx, int instance, int what, double* out) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, IB_PF_E_ARG, "bad instance");
  if (!out) return fail(ctx, IB_PF_E_ARG, "null output");
  Instance& in = ctx->inst[instance];
  switch (what) {
    case IB_PF_Q_MASS: {
      CK(join_in(*ctx));
      mass_reduce(in, ctx->precision, in.C[ctx->cur], in.Clo[ctx->cur], ctx->work);
      CK(cudaGetLastError());
      double m = 0;
      CK(cudaMemcpyAsync(&m, in.mass, sizeof(double), cudaMemcpyDeviceToHost, ctx->work));
      CK(cudaStreamSynchronize(ctx->work));
      *out = m;
      return IB_PF_OK;
    }
    case IB_PF_Q_N_GHOST: *out = in.tab.ng; return IB_PF_OK;
    case IB_PF_Q_N_FACE_U: *out = in.tab.nfu; return IB_PF_OK;
    case IB_PF_Q_N_FACE_V: *out = in.tab.nfv; return IB_PF_OK;
    case IB_PF_Q_N_FACE_W: *out = in.tab.nfw; return IB_PF_OK;
    case IB_PF_Q_STATUS: {
      CK(join_in(*ctx));
      int s = 0;
      CK(cudaMemcpyAsync(&s, in.status, sizeof(int), cudaMemcpyDeviceToHost, ctx->work));
      CK(cudaStreamSynchronize(ctx->work));
      *out = s;
      return IB_PF_OK;
    }
    case IB_PF_Q_STEPS: *out = (double)ctx->steps; return IB_PF_OK;
    case IB_PF_Q_N_FALLBACK: *out = in.tab.n_fallback; return IB_PF_OK;
    case IB_PF_Q_LAUNCHES_PER_STEP: {
      ib_pf_status st = ctx->weights_ready ? capture_graphs(ctx) : IB_PF_E_STATE;
      if (st != IB_PF_OK) return fail(ctx, st, "launch count needs the precompute");
      *out = ctx->launches_per_step;
      return IB_PF_OK;
    }
    default: return fail(ctx, IB_PF_E_ARG, "bad query id");
  }
}

ib_pf_status ib_pf_set_kernel_timing(ib_pf_ctx* ctx, int enable) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  const bool want = enable != 0;
  if (want == ctx->timing) return IB_PF_OK;
  CK(cudaStreamSynchronize(ctx->work));
  for (int ph = 0; ph < 2; ++ph) {
    if (ctx->graph[ph]) cudaGraphExecDestroy(ctx->graph[ph]);
    ctx->graph[ph] = nullptr;
  }
  ctx->timing = want;
  return IB_PF_OK;
}

namespace {
// the tile row widths built for a transform of 2^logn points
bool tile_rb_built(int logn, int rb) { return (rb == 128 && logn <= 9) || (rb == 64 && logn >= 8); }

void drop_graphs(ib_pf_ctx* ctx) {
  for (int ph = 0; ph < 2; ++ph) {
    if (ctx->graph[ph]) cudaGraphExecDestroy(ctx->graph[ph]);
    ctx->graph[ph] = nullptr;
  }
}
}  // namespace

ib_pf_status ib_pf_set_tuning(ib_pf_ctx* ctx, int instance, const ib_pf_tuning* t) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (!t) return fail(ctx, IB_PF_E_ARG, "null tuning");
  if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, IB_PF_E_ARG, "instance out of range");
  Instance& in = ctx->inst[instance];
  if (in.dim != 3) return fail(ctx, IB_PF_E_UNSUPPORTED, "tuning applies to 3D instances");
  if (t->y_tile_bytes != 0 && !tile_rb_built(in.logny, t->y_tile_bytes))
    return fail(ctx, IB_PF_E_ARG, "y_tile_bytes not built for ny");
  if (t->z_tile_bytes != 0 && !tile_rb_built(in.lognz, t->z_tile_bytes))
    return fail(ctx, IB_PF_E_ARG, "z_tile_bytes not built for nz");
  const int pp = t->predict_planes;
  if (pp != 0 && pp != 8 && pp != 16 && pp != 32) return fail(ctx, IB_PF_E_ARG, "predict_planes must be 0, 8, 16 or 32");
  CK(cudaStreamSynchronize(ctx->work));
  in.tune_y_rb = t->y_tile_bytes;
  in.tune_z_rb = t->z_tile_bytes;
  in.tune_pred_planes = pp;
  drop_graphs(ctx);
  return IB_PF_OK;
}

ib_pf_status ib_pf_get_tuning(ib_pf_ctx* ctx, int instance, ib_pf_tuning* t) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (!t) return fail(ctx, IB_PF_E_ARG, "null tuning");
  if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, IB_PF_E_ARG, "instance out of range");
  const Instance& in = ctx->inst[instance];
  t->y_tile_bytes = in.tune_y_rb;
  t->z_tile_bytes = in.tune_z_rb;
  t->predict_planes = in.tune_pred_planes;
  return IB_PF_OK;
}

ib_pf_status ib_pf_autotune(ib_pf_ctx* ctx, int instance, int reps, ib_pf_tuning* chosen,
                            double* times_ms) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, IB_PF_E_ARG, "instance out of range");
  if (reps < 1) return fail(ctx, IB_PF_E_ARG, "reps < 1");
  Instance& in = ctx->inst[instance];
  if (in.dim != 3) return fail(ctx, IB_PF_E_UNSUPPORTED, "tuning applies to 3D instances");
  if (!ctx->weights_ready) return fail(ctx, IB_PF_E_STATE, "ib_pf_precompute_weights has not succeeded");
  CK(cudaStreamSynchronize(ctx->work));
  float t[7];
  const int rbs[2] = {128, 64}, planes[3] = {8, 16, 32};
  for (int q = 0; q < 2; ++q) t[q] = spectral3_time_tiles(in, ctx->precision, 1, rbs[q], reps, ctx->work);
  for (int q = 0; q < 2; ++q) t[2 + q] = spectral3_time_tiles(in, ctx->precision, 2, rbs[q], reps, ctx->work);
  for (int q = 0; q < 3; ++q)
    t[4 + q] = planes[q] <= in.nz || q == 0 ? step3d_time_predict(*ctx, in, planes[q], reps, ctx->work) : -1.0f;
  CK(cudaGetLastError());
  auto best = [&](int first, int n, const int* vals) {
    int b = -1;
    for (int q = 0; q < n; ++q)
      if (t[first + q] >= 0.0f && (b < 0 || t[first + q] < t[first + b])) b = q;
    return b < 0 ? 0 : vals[b];
  };
  ib_pf_tuning tu;
  tu.y_tile_bytes = best(0, 2, rbs);
  tu.z_tile_bytes = best(2, 2, rbs);
  tu.predict_planes = best(4, 3, planes);
  if (times_ms)
    for (int q = 0; q < 7; ++q) times_ms[q] = (double)t[q];
  if (chosen) *chosen = tu;
  return ib_pf_set_tuning(ctx, instance, &tu);
}

ib_pf_status ib_pf_kernel_times(ib_pf_ctx* ctx, int cap, double* ms, const char** names, int* n) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (!ctx->timing || ctx->steps == 0 || ctx->tev.size() < 2)
    return fail(ctx, IB_PF_E_STATE, "no timed step: call ib_pf_set_kernel_timing(ctx, 1) and step");
  CK(cudaStreamSynchronize(ctx->work));
  const int nk = (int)ctx->tnames.size();
  if (n) *n = nk;
  for (int k = 0; k < nk && k < cap; ++k) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, ctx->tev[k], ctx->tev[k + 1]));
    if (ms) ms[k] = (double)t;
    if (names) names[k] = ctx->tnames[k];
  }
  return IB_PF_OK;
}

ib_pf_status ib_pf_bind_fields(ib_pf_ctx* ctx, int instance, int field_id, int time_level,
                               void* device_ptr, long long nbytes) {
  if (!ctx) return fail(nullptr, IB_PF_E_ARG, "null context");
  if (instance < 0 || instance >= (int)ctx->inst.size()) return fail(ctx, IB_PF_E_ARG, "bad instance");
  Instance& in = ctx->inst[instance];
  void** slot = nullptr;
  const int lv = time_level == 0 ? ctx->cur : 1 - ctx->cur;
  const bool two = time_level == 0 || time_level == 1;
  switch (field_id) {
    case IB_PF_F_C: slot = two ? &in.C[lv] : nullptr; break;
    case IB_PF_F_U: slot = two ? &in.U[lv] : nullptr; break;
    case IB_PF_F_V: slot = two ? &in.V[lv] : nullptr; break;
    case IB_PF_F_P: slot = two ? &in.P[lv] : nullptr; break;
    case IB_PF_F_W: slot = (two && in.dim == 3) ? &in.W[lv] : nullptr; break;
    case IB_PF_F_C_LO: slot = (two && ctx->precision == IB_PF_FP32) ? &in.Clo[lv] : nullptr; break;
    case IB_PF_F_HU: slot = time_level == 0 ? &in.Hu : nullptr; break;
    case IB_PF_F_HV: slot = time_level == 0 ? &in.Hv : nullptr; break;
    case IB_PF_F_HW: slot = (time_level == 0 && in.dim == 3) ? &in.Hw : nullptr; break;
    default: break;
  }
  if (!slot) return fail(ctx, IB_PF_E_ARG, "field id / time level cannot be bound");
  if (!device_ptr) return fail(ctx, IB_PF_E_ARG, "null device pointer");
  if (((uintptr_t)device_ptr & 15u) != 0) return fail(ctx, IB_PF_E_ARG, "device pointer not 16-byte aligned");
  const size_t want = field_elems(in, field_id) * ctx->esz;
  if (nbytes != (long long)want)
    return fail(ctx, IB_PF_E_ARG, "nbytes " + std::to_string(nbytes) + " != field size " + std::to_string(want));
  cudaPointerAttributes pa;
  CK(cudaPointerGetAttributes(&pa, device_ptr));
  if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
    return fail(ctx, IB_PF_E_ARG, "not device memory");
  for (Instance& other : ctx->inst)
    for (void** q : {&other.C[0], &other.C[1], &other.U[0], &other.U[1], &other.V[0], &other.V[1],
                     &other.P[0], &other.P[1], &other.W[0], &other.W[1], &other.Clo[0], &other.Clo[1],
                     &other.Hu, &other.Hv, &other.Hw})
      if (q != slot && *q == device_ptr) return fail(ctx, IB_PF_E_ARG, "buffer already bound to another field");
  CK(cudaStreamSynchronize(ctx->work));
  void* old = *slot;
  bool old_bound = false;
  for (void* b : in.bound) old_bound = old_bound || b == old;
  if (old && !old_bound) CK(cudaFree(old));
  if (old_bound)
    for (void*& b : in.bound)
      if (b == old) b = nullptr;
  *slot = device_ptr;
  in.bound.push_back(device_ptr);
  // the wall rows (planes) of v (w) stay zero
  const size_t nxy = (size_t)in.nx * in.ny;
  if (field_id == IB_PF_F_V && in.dim == 2) {
    CK(cudaMemsetAsync(device_ptr, 0, (size_t)in.nx * ctx->esz, ctx->work));
    CK(cudaMemsetAsync((char*)device_ptr + (size_t)in.ny * in.nx * ctx->esz, 0, (size_t)in.nx * ctx->esz, ctx->work));
  }
  if (field_id == IB_PF_F_W) {
    CK(cudaMemsetAsync(device_ptr, 0, nxy * ctx->esz, ctx->work));
    CK(cudaMemsetAsync((char*)device_ptr + (size_t)in.nz * nxy * ctx->esz, 0, nxy * ctx->esz, ctx->work));
  }
  // the step graphs (and, in 2D, the device descriptors of the batched launches) hold the
  // field pointers: rebuild them
  for (int ph = 0; ph < 2; ++ph) {
    if (ctx->graph[ph]) cudaGraphExecDestroy(ctx->graph[ph]);
    ctx->graph[ph] = nullptr;
  }
  if (ctx->plan) {
    batch_free(*(BatchPlan*)ctx->plan);
    CK(batch_setup(*ctx, *(BatchPlan*)ctx->plan));
  }
  CK(cudaStreamSynchronize(ctx->work));
  return IB_PF_OK;
}

const char* ib_pf_last_error(const ib_pf_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void ib_pf_destroy(ib_pf_ctx* ctx) {
  if (!ctx) return;
  if (ctx->work) cudaStreamSynchronize(ctx->work);
  for (int ph = 0; ph < 2; ++ph)
    if (ctx->graph[ph]) cudaGraphExecDestroy(ctx->graph[ph]);
  for (Instance& in : ctx->inst) free_instance(in);
  if (ctx->plan) {
    batch_free(*(BatchPlan*)ctx->plan);
    delete (BatchPlan*)ctx->plan;
  }
  for (cudaEvent_t e : ctx->tev) cudaEventDestroy(e);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->work) cudaStreamDestroy(ctx->work);
  delete ctx;
}

}  // extern "C"
