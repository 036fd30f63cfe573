"""Thin ctypes binding of the ib_pf C ABI (include/ib_pf.h).

Argument marshalling only: every step of the method runs in the CUDA library.  The
functions below carry the C names; ``Solver`` bundles them for one context.  Loading
fails loudly (``ImportError``/``OSError``) when the compiled library is missing: there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes as ct
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_lib" / "libibpf.so"

# ---- enums (mirror include/ib_pf.h)
OK, E_ARG, E_UNSUPPORTED, E_CUDA, E_NUMERIC, E_TIMEOUT, E_STATE, E_GEOMETRY = 0, -1, -2, -3, -4, -5, -6, -7
FP64, FP32, FP32_3XBF16 = 0, 1, 2   # ib_pf_precision
CH_SEMI_IMPLICIT, CH_EXPLICIT = 0, 1
W_LINEAR, W_IDW = 0, 1            # ib_pf_weights
NS_EXPLICIT, NS_SEMI_IMPLICIT = 0, 1   # ib_pf_ns_scheme
WALL_FLAT, WALL_SINUSOID, WALL_NONE, WALL_SPHERE, WALL_SPHERES, WALL_MASK = 0, 1, 3, 4, 5, 6
(F_C, F_C_OLD, F_U, F_U_OLD, F_V, F_V_OLD, F_HU, F_HV, F_P, F_P_OLD, F_PHI, F_Q, F_RHS_P,
 F_C_LO, F_C_OLD_LO, F_W, F_W_OLD, F_HW, F_C_I) = range(19)
FIELD_IDS = {"C": F_C, "C_old": F_C_OLD, "u": F_U, "u_old": F_U_OLD, "v": F_V, "v_old": F_V_OLD,
             "Hu": F_HU, "Hv": F_HV, "P": F_P, "P_old": F_P_OLD, "phi": F_PHI, "Q": F_Q,
             "rhs_p": F_RHS_P, "C_lo": F_C_LO, "C_old_lo": F_C_OLD_LO, "w": F_W,
             "w_old": F_W_OLD, "Hw": F_HW, "C_I": F_C_I}
STATE_FIELDS = ("C", "C_old", "u", "u_old", "v", "v_old", "Hu", "Hv", "P", "P_old")
STATE_FIELDS_3D = STATE_FIELDS + ("w", "w_old", "Hw")
(T_ALPHA_C, T_ALPHA_U, T_ALPHA_V, T_CLASS, T_GHOST_CELL, T_NORMAL, T_DN, T_GAMMA, T_AP1, T_W1,
 T_AP2, T_W2, T_FACE_U, T_FACE_V, T_ALPHA_W, T_FACE_W) = range(16)
_TABLE_DTYPE = {T_ALPHA_C: np.float64, T_ALPHA_U: np.float64, T_ALPHA_V: np.float64,
                T_CLASS: np.int32, T_GHOST_CELL: np.int32, T_NORMAL: np.float64,
                T_DN: np.float64, T_GAMMA: np.float64, T_AP1: np.int32, T_W1: np.float64,
                T_AP2: np.int32, T_W2: np.float64, T_FACE_U: np.int32, T_FACE_V: np.int32,
                T_ALPHA_W: np.float64, T_FACE_W: np.int32}
(Q_MASS, Q_N_GHOST, Q_N_FACE_U, Q_N_FACE_V, Q_STATUS, Q_STEPS, Q_N_FALLBACK, Q_LAUNCHES,
 Q_N_FACE_W) = range(9)


class Grid(ct.Structure):
    _fields_ = [("dim", ct.c_int), ("n", ct.c_int * 3), ("L", ct.c_double * 3)]


class Geometry(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("p", ct.c_double * 8),
                ("spheres", ct.POINTER(ct.c_double)), ("n_spheres", ct.c_int),
                ("alpha", ct.POINTER(ct.c_double))]


PARAM_NAMES = ("Re", "Ca", "Cn", "Pe", "S", "rho_ratio", "mu_ratio", "theta_deg", "l_s", "mu_f",
               "d1", "d2", "dt")


class Params(ct.Structure):
    _fields_ = [(n, ct.c_double) for n in PARAM_NAMES] + [("precision", ct.c_int), ("ch_scheme", ct.c_int),
                                                         ("weights", ct.c_int), ("ns_scheme", ct.c_int)]


class Tuning(ct.Structure):
    _fields_ = [("y_tile_bytes", ct.c_int), ("z_tile_bytes", ct.c_int), ("predict_planes", ct.c_int)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


TUNING_CANDIDATES = ("y128", "y64", "z128", "z64", "planes8", "planes16", "planes32")


class IbPfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ib_pf status {status}: {msg}")
        self.status = status


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"ib_pf CUDA library not built: {_LIB_PATH} is missing "
                          "(run __graft_entry__.build())")
    lib = ct.CDLL(str(_LIB_PATH))
    vp, i, ll = ct.c_void_p, ct.c_int, ct.c_longlong
    sigs = {
        "ib_pf_init_geometry": (i, [ct.POINTER(vp), i, ct.POINTER(Grid), ct.POINTER(Geometry),
                                    ct.POINTER(Params), vp]),
        "ib_pf_precompute_weights": (i, [vp]),
        "ib_pf_step": (i, [vp, i]),
        "ib_pf_read_fields": (i, [vp, i, i, vp, ll, i]),
        "ib_pf_write_fields": (i, [vp, i, i, vp, ll, i]),
        "ib_pf_write_fields_batch": (i, [vp, i, ct.POINTER(i), ct.POINTER(i), ct.POINTER(vp),
                                         ct.POINTER(ll), i]),
        "ib_pf_read_fields_batch": (i, [vp, i, ct.POINTER(i), ct.POINTER(i), ct.POINTER(vp),
                                        ct.POINTER(ll), i]),
        "ib_pf_read_table": (i, [vp, i, i, vp, ll, ct.POINTER(ll)]),
        "ib_pf_query": (i, [vp, i, i, ct.POINTER(ct.c_double)]),
        "ib_pf_set_kernel_timing": (i, [vp, i]),
        "ib_pf_kernel_times": (i, [vp, i, ct.POINTER(ct.c_double), ct.POINTER(ct.c_char_p),
                                   ct.POINTER(i)]),
        "ib_pf_poisson_solve_noalloc": (i, [vp, vp, i, i, ct.c_double, vp]),
        "ib_pf_bind_fields": (i, [vp, i, i, i, vp, ct.c_longlong]),
        "ib_pf_set_tuning": (i, [vp, i, ct.POINTER(Tuning)]),
        "ib_pf_get_tuning": (i, [vp, i, ct.POINTER(Tuning)]),
        "ib_pf_autotune": (i, [vp, i, i, ct.POINTER(Tuning), ct.POINTER(ct.c_double)]),
        "ib_pf_last_error": (ct.c_char_p, [vp]),
        "ib_pf_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load()
    return _lib


def library_path() -> Path:
    return _LIB_PATH


# ---- C-named wrappers -----------------------------------------------------------
def ib_pf_last_error(ctx) -> str:
    s = lib().ib_pf_last_error(ctx)
    return s.decode() if s else ""


def _check(st: int, ctx=None):
    if st != OK:
        raise IbPfError(st, ib_pf_last_error(ctx))


def ib_pf_init_geometry(grids, geoms, params, stream: int = 0):
    n = len(grids)
    G = (Grid * n)(*grids)
    W = (Geometry * n)(*geoms)
    P = (Params * n)(*params)
    out = ct.c_void_p()
    _check(lib().ib_pf_init_geometry(ct.byref(out), n, G, W, P, ct.c_void_p(stream)))
    return out


def ib_pf_precompute_weights(ctx):
    _check(lib().ib_pf_precompute_weights(ctx), ctx)


def ib_pf_step(ctx, nsteps: int):
    _check(lib().ib_pf_step(ctx, int(nsteps)), ctx)


def ib_pf_read_fields(ctx, instance: int, field_id: int, dst_ptr: int, nbytes: int, dst_on_host: bool):
    _check(lib().ib_pf_read_fields(ctx, instance, field_id, ct.c_void_p(dst_ptr), nbytes,
                                   int(dst_on_host)), ctx)


def ib_pf_write_fields(ctx, instance: int, field_id: int, src_ptr: int, nbytes: int, src_on_host: bool):
    _check(lib().ib_pf_write_fields(ctx, instance, field_id, ct.c_void_p(src_ptr), nbytes,
                                    int(src_on_host)), ctx)


def _batch_args(items):
    n = len(items)
    inst = (ct.c_int * n)(*[it[0] for it in items])
    fids = (ct.c_int * n)(*[it[1] for it in items])
    ptrs = (ct.c_void_p * n)(*[it[2] for it in items])
    nb = (ct.c_longlong * n)(*[it[3] for it in items])
    return n, inst, fids, ptrs, nb


def ib_pf_write_fields_batch(ctx, items, src_on_host: bool):
    """items: (instance, field_id, src_ptr, nbytes) tuples."""
    n, inst, fids, ptrs, nb = _batch_args(items)
    _check(lib().ib_pf_write_fields_batch(ctx, n, inst, fids, ptrs, nb, int(src_on_host)), ctx)


def ib_pf_read_fields_batch(ctx, items, dst_on_host: bool):
    """items: (instance, field_id, dst_ptr, nbytes) tuples."""
    n, inst, fids, ptrs, nb = _batch_args(items)
    _check(lib().ib_pf_read_fields_batch(ctx, n, inst, fids, ptrs, nb, int(dst_on_host)), ctx)


def ib_pf_read_table(ctx, instance: int, table_id: int, dst_ptr: int | None, nbytes: int) -> int:
    cnt = ct.c_longlong(0)
    _check(lib().ib_pf_read_table(ctx, instance, table_id, ct.c_void_p(dst_ptr or 0), nbytes,
                                  ct.byref(cnt)), ctx)
    return cnt.value


def ib_pf_query(ctx, instance: int, what: int) -> float:
    out = ct.c_double(0.0)
    _check(lib().ib_pf_query(ctx, instance, what, ct.byref(out)), ctx)
    return out.value


def ib_pf_set_kernel_timing(ctx, enable: bool):
    _check(lib().ib_pf_set_kernel_timing(ctx, int(enable)), ctx)


def ib_pf_kernel_times(ctx, cap: int = 4096):
    ms = (ct.c_double * cap)()
    names = (ct.c_char_p * cap)()
    n = ct.c_int(0)
    _check(lib().ib_pf_kernel_times(ctx, cap, ms, names, ct.byref(n)), ctx)
    k = min(n.value, cap)
    return [names[i].decode() for i in range(k)], [ms[i] for i in range(k)]


def ib_pf_bind_fields(ctx, instance: int, field_id: int, time_level: int, device_ptr: int,
                      nbytes: int):
    _check(lib().ib_pf_bind_fields(ctx, instance, field_id, time_level, ct.c_void_p(device_ptr),
                                   nbytes), ctx)


def ib_pf_set_tuning(ctx, instance: int, tuning: Tuning):
    _check(lib().ib_pf_set_tuning(ctx, instance, ct.byref(tuning)), ctx)


def ib_pf_get_tuning(ctx, instance: int) -> Tuning:
    t = Tuning()
    _check(lib().ib_pf_get_tuning(ctx, instance, ct.byref(t)), ctx)
    return t


def ib_pf_autotune(ctx, instance: int, reps: int):
    t = Tuning()
    ms = (ct.c_double * len(TUNING_CANDIDATES))()
    _check(lib().ib_pf_autotune(ctx, instance, reps, ct.byref(t), ms), ctx)
    return t, dict(zip(TUNING_CANDIDATES, list(ms)))


def ib_pf_poisson_solve_noalloc(rhs_ptr: int, out_ptr: int, nx: int, ny: int, h: float,
                                stream: int = 0):
    _check(lib().ib_pf_poisson_solve_noalloc(ct.c_void_p(rhs_ptr), ct.c_void_p(out_ptr), nx, ny,
                                             float(h), ct.c_void_p(stream)))


def ib_pf_destroy(ctx):
    lib().ib_pf_destroy(ctx)


# ---- convenience --------------------------------------------------------------------
def make_grid(nx: int, ny: int, lx: float, ly: float) -> Grid:
    g = Grid()
    g.dim = 2
    g.n[0], g.n[1], g.n[2] = nx, ny, 1
    g.L[0], g.L[1], g.L[2] = lx, ly, 0.0
    return g


def make_grid3(nx: int, ny: int, nz: int, lx: float, ly: float, lz: float) -> Grid:
    g = Grid()
    g.dim = 3
    g.n[0], g.n[1], g.n[2] = nx, ny, nz
    g.L[0], g.L[1], g.L[2] = lx, ly, lz
    return g


def make_geometry(kind: int, p, spheres=(), alpha=()) -> Geometry:
    """spheres: (cx, cy, cz, r) rows for WALL_SPHERES; alpha: the volume-fraction arrays of
    WALL_MASK (alpha_c, alpha_u, alpha_v[, alpha_w]), concatenated here.  The arrays stay
    referenced by the returned object, and ib_pf_init_geometry copies them."""
    w = Geometry()
    w.kind = kind
    for k, x in enumerate(p):
        w.p[k] = float(x)
    keep = []
    if len(spheres):
        arr = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
        keep.append(arr)
        w.spheres = arr.ctypes.data_as(ct.POINTER(ct.c_double))
        w.n_spheres = arr.shape[0]
    if len(alpha):
        arr = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in alpha]))
        keep.append(arr)
        w.alpha = arr.ctypes.data_as(ct.POINTER(ct.c_double))
    w._keep = keep
    return w


def make_params(precision: int = FP64, ch_scheme: int = CH_SEMI_IMPLICIT, weights: int = 0,
                ns_scheme: int = 0, **kw) -> Params:
    p = Params()
    for n in PARAM_NAMES:
        setattr(p, n, float(kw[n]))
    p.precision = precision
    p.ch_scheme = int(ch_scheme)
    p.weights = int(weights)
    p.ns_scheme = int(ns_scheme)
    return p


class Solver:
    """One ib_pf context.  Field I/O accepts numpy arrays (host) or torch CUDA tensors."""

    def __init__(self, grids, geoms, params, stream: int = 0):
        self.ctx = ib_pf_init_geometry(grids, geoms, params, stream)
        self.precision = params[0].precision
        self.dtype = np.float64 if self.precision == FP64 else np.float32
        self.dim = grids[0].dim
        self.shapes = [(g.n[2], g.n[1], g.n[0]) if g.dim == 3 else (g.n[1], g.n[0]) for g in grids]
        self.state_fields = STATE_FIELDS_3D if self.dim == 3 else STATE_FIELDS
        self.dynamic = any(p.mu_f > 0.0 for p in params)

    def close(self):
        if self.ctx:
            ib_pf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field_dtype(self, name: str):
        """Element type of a field: the context's, except the FP64 wall values C_I."""
        return np.float64 if name == "C_I" else self.dtype

    def field_shape(self, name: str, instance: int = 0):
        if name == "C_I":
            return (int(self.query(Q_N_GHOST, instance)),)
        if self.dim == 3:
            nz, ny, nx = self.shapes[instance]
            return (nz + 1, ny, nx) if name in ("w", "w_old", "Hw") else (nz, ny, nx)
        ny, nx = self.shapes[instance]
        return (ny + 1, nx) if name in ("v", "v_old", "Hv") else (ny, nx)

    def bind(self, name: str, tensor, time_level: int = 0, instance: int = 0):
        """Make a contiguous torch CUDA tensor the storage of a state field (ib_pf_bind_fields);
        the tensor must outlive the context (a reference is kept here)."""
        assert tensor.is_cuda and tensor.is_contiguous()
        ib_pf_bind_fields(self.ctx, instance, FIELD_IDS[name], time_level, tensor.data_ptr(),
                          tensor.numel() * tensor.element_size())
        self._bound = getattr(self, "_bound", []) + [tensor]

    def precompute_weights(self):
        ib_pf_precompute_weights(self.ctx)

    def tuning(self, instance: int = 0) -> dict:
        return ib_pf_get_tuning(self.ctx, instance).as_dict()

    def set_tuning(self, instance: int = 0, **choice):
        t = Tuning(**{k: int(choice.get(k, 0)) for k, _ in Tuning._fields_})
        ib_pf_set_tuning(self.ctx, instance, t)

    def autotune(self, instance: int = 0, reps: int = 3, cache: str | Path | None = None,
                 gpu_name: str | None = None) -> dict:
        """The 3D schedule of `instance`: taken from the JSON file `cache` when it holds an
        entry for this grid shape, precision and GPU, else timed by ib_pf_autotune (state
        unchanged) and written there.  Returns the choice, plus the candidates' times when
        they were measured."""
        import json
        n = self.shapes[instance]
        if gpu_name is None:
            try:
                import torch
                gpu_name = torch.cuda.get_device_name()
            except Exception:   # no torch / no device name: key without it
                gpu_name = "unknown"
        form = {FP64: 'fp64', FP32: 'fp32', FP32_3XBF16: 'fp32_3xbf16'}[self.precision]
        key = "x".join(str(v) for v in n[::-1]) + f":{form}:{gpu_name}"
        table = {}
        if cache is not None and Path(cache).exists():
            table = json.loads(Path(cache).read_text())
        if key in table:
            self.set_tuning(instance, **table[key]["choice"])
            return {"key": key, "choice": table[key]["choice"], "cached": True}
        t, ms = ib_pf_autotune(self.ctx, instance, reps)
        entry = {"choice": t.as_dict(), "ms": ms}
        if cache is not None:
            table[key] = entry
            Path(cache).write_text(json.dumps(table, indent=1, sort_keys=True))
        return {"key": key, "cached": False, **entry}

    def step(self, nsteps: int = 1):
        ib_pf_step(self.ctx, nsteps)

    def write(self, name: str, arr, instance: int = 0):
        if hasattr(arr, "data_ptr"):   # torch tensor (device, or pinned host memory)
            assert arr.is_contiguous()
            ib_pf_write_fields(self.ctx, instance, FIELD_IDS[name], arr.data_ptr(),
                               arr.numel() * arr.element_size(), not arr.is_cuda)
            return
        a = np.ascontiguousarray(arr, dtype=self.field_dtype(name))
        assert a.shape == self.field_shape(name, instance), (name, a.shape)
        ib_pf_write_fields(self.ctx, instance, FIELD_IDS[name], a.ctypes.data, a.nbytes, True)

    def read(self, name: str, instance: int = 0, out=None) -> np.ndarray:
        if out is not None and hasattr(out, "data_ptr"):
            ib_pf_read_fields(self.ctx, instance, FIELD_IDS[name], out.data_ptr(),
                              out.numel() * out.element_size(), not out.is_cuda)
            return out
        a = np.empty(self.field_shape(name, instance), dtype=self.field_dtype(name))
        ib_pf_read_fields(self.ctx, instance, FIELD_IDS[name], a.ctypes.data, a.nbytes, True)
        return a

    def prepare_writes(self, items) -> "FieldBatch":
        """A reusable batched write of (name, array, instance) items (torch tensors or
        contiguous numpy arrays of the context's dtype, all on the host or all on the device):
        the argument arrays are built once; .run() issues the one C call."""
        return FieldBatch(self, items, write=True)

    def prepare_reads(self, items) -> "FieldBatch":
        """The same for batched reads into preallocated (name, out, instance) buffers."""
        return FieldBatch(self, items, write=False)

    def write_many(self, items):
        """items: (name, array, instance) with numpy host arrays or torch tensors, all on
        the host or all on the device; one synchronisation for the whole batch."""
        items = [(n, a if hasattr(a, "data_ptr") else np.ascontiguousarray(a, dtype=self.dtype), k)
                 for n, a, k in items]
        if items:
            FieldBatch(self, items, write=True).run()

    def read_many(self, items):
        """items: (name, out, instance) with preallocated numpy arrays or torch tensors, all on
        the host or all on the device; one synchronisation for the whole batch."""
        if items:
            FieldBatch(self, list(items), write=False).run()

    def table(self, table_id: int, instance: int = 0) -> np.ndarray:
        n = ib_pf_read_table(self.ctx, instance, table_id, None, 0)
        a = np.empty(n, dtype=_TABLE_DTYPE[table_id])
        if n:
            ib_pf_read_table(self.ctx, instance, table_id, a.ctypes.data, a.nbytes)
        return a

    def query(self, what: int, instance: int = 0) -> float:
        return ib_pf_query(self.ctx, instance, what)

    def write_state(self, state: dict, instance: int = 0):
        for name in self.state_fields:
            self.write(name, state[name], instance)

    def read_state(self, instance: int = 0) -> dict:
        return {name: self.read(name, instance) for name in self.state_fields}

    def read_checkpoint(self, instance: int = 0) -> dict:
        """Everything needed for a bit-exact restart (state plus, in FP32 contexts, the
        low parts of the compensated C)."""
        d = self.read_state(instance)
        if self.precision != FP64:
            d["C_lo"] = self.read("C_lo", instance)
            d["C_old_lo"] = self.read("C_old_lo", instance)
        if self.dynamic:
            d["C_I"] = self.read("C_I", instance)
        return d

    def write_checkpoint(self, d: dict, instance: int = 0):
        self.write_state(d, instance)
        for name in ("C_lo", "C_old_lo", "C_I"):
            if name in d:
                self.write(name, d[name], instance)


class FieldBatch:
    """Prepared arguments of one batched field read or write (see Solver.prepare_writes)."""

    def __init__(self, solver: Solver, items, write: bool):
        self.solver, self.write = solver, write
        self._keep = []
        args, host = [], None
        for name, arr, inst in items:
            if hasattr(arr, "data_ptr"):
                assert arr.is_contiguous()
                on_host = not arr.is_cuda
                ptr, nb = arr.data_ptr(), arr.numel() * arr.element_size()
            else:
                assert arr.flags["C_CONTIGUOUS"] and arr.dtype == solver.dtype
                on_host, ptr, nb = True, arr.ctypes.data, arr.nbytes
            self._keep.append(arr)
            assert host is None or host == on_host, "mixed host and device buffers"
            host = on_host
            args.append((inst, FIELD_IDS[name], ptr, nb))
        self.on_host = bool(host)
        self.n, self.inst, self.fids, self.ptrs, self.nb = _batch_args(args)

    def run(self):
        fn = lib().ib_pf_write_fields_batch if self.write else lib().ib_pf_read_fields_batch
        _check(fn(self.solver.ctx, self.n, self.inst, self.fids, self.ptrs, self.nb,
                  int(self.on_host)), self.solver.ctx)


def solver_from_cases(cases, precision: int = FP64, stream: int = 0) -> Solver:
    """Build a Solver from objects carrying nx, ny, lx, ly (and nz, lz, spheres in 3D),
    geom_kind, geom_p and a ``params`` object with the ib_pf_params fields (duck-typed; no
    import of callers)."""
    grids = [make_grid3(c.nx, c.ny, c.nz, c.lx, c.ly, c.lz) if hasattr(c, "nz")
             else make_grid(c.nx, c.ny, c.lx, c.ly) for c in cases]
    geoms = [make_geometry(c.geom_kind, c.geom_p, getattr(c, "spheres", ()), getattr(c, "alpha", ()))
             for c in cases]
    params = [make_params(precision, getattr(c.params, "ch_scheme", CH_SEMI_IMPLICIT),
                          getattr(c.params, "weights", W_LINEAR),
                          getattr(c.params, "ns_scheme", NS_EXPLICIT),
                          **{n: getattr(c.params, n) for n in PARAM_NAMES}) for c in cases]
    return Solver(grids, geoms, params, stream)
