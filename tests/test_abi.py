"""C-ABI library checks that need no GPU: it builds, loads, exports every entry point
declared in include/ib_pf.h, and rejects invalid arguments before touching the device."""
import ctypes as ct
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "ib_pf.h"


def _declared():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ib_pf_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf
    return ibpf


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ib_pf_init_geometry", "ib_pf_precompute_weights", "ib_pf_step",
              "ib_pf_read_fields"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    so = ct.CDLL(str(lib.library_path()))
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def _args(lib, nx=128, ny=64, **over):
    kw = dict(Re=10.0, Ca=0.1, Cn=0.02, Pe=5e3, S=2.0, rho_ratio=10.0, mu_ratio=10.0,
              theta_deg=60.0, l_s=0.0, mu_f=0.0, d1=2 ** 0.5 / 64, d2=2 ** 0.5 / 128, dt=1e-4)
    kw.update(over)
    return ([lib.make_grid(nx, ny, 2.0, 1.0)], [lib.make_geometry(lib.WALL_FLAT, [0.1])],
            [lib.make_params(lib.FP64, **kw)])


@pytest.mark.parametrize("bad,status", [
    (dict(nx=100), -1),                 # not a power of two
    (dict(ny=4), -1),                   # too small
    (dict(Cn=-1.0), -1),                # negative parameter
    (dict(mu_f=-0.5), -1),              # negative wall friction
    (dict(weights=7), -1),              # unknown averaging weights
    (dict(ns_scheme=5), -1),            # unknown momentum predictor
    (dict(d1=0.001), -1),               # d1 not beyond half a cell diagonal
])
def test_invalid_arguments_rejected_on_host(lib, bad, status):
    nx = bad.pop("nx", 128)
    ny = bad.pop("ny", 64)
    g, w, p = _args(lib, nx=nx, ny=ny, **bad)
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g, w, p)
    assert ei.value.status == status
    assert lib.ib_pf_last_error(None)


def _args3(lib, n=(32, 32, 32), L=(1.0, 1.0, 1.0), kind=None, p=(0.5, 0.5, 0.5, 0.25),
            spheres=(), d1=None):
    from workloads import cases as W
    c = W.small_sphere_case(32)
    g = lib.make_grid3(*n, *L)
    w = lib.make_geometry(lib.WALL_SPHERE if kind is None else kind, p, spheres)
    kw = {k: getattr(c.params, k) for k in lib.PARAM_NAMES}
    if d1 is not None:
        kw["d1"] = d1
    return [g], [w], [lib.make_params(lib.FP64, **kw)]


@pytest.mark.parametrize("bad", [
    {"n": (32, 32, 12)},                       # not a power of two
    {"n": (2048, 32, 32)},                     # beyond the 3D limit
    {"L": (1.0, 2.0, 1.0)},                    # non-cubic cells
    {"kind": 1},                               # the sinusoidal wall is 2D only
    {"p": (0.5, 0.5, 0.5, 0.0)},               # zero sphere radius
    {"kind": 5},                               # SPHERES without spheres
    {"kind": 5, "spheres": [(0.5, 0.5, 0.2, -0.1)]},
    {"d1": 0.8 * 0.5 * 3 ** 0.5 / 32},         # d1 below half the 3D cell diagonal
])
def test_invalid_3d_arguments_rejected_on_host(lib, bad):
    g, w, p = _args3(lib, **bad)
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g, w, p)
    assert ei.value.status == lib.E_ARG
    assert lib.ib_pf_last_error(None)


def test_mixed_dimensions_rejected(lib):
    g2, w2, p2 = _args(lib)
    g3, w3, p3 = _args3(lib)
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g2 + g3, w2 + w3, p2 + p3)
    assert ei.value.status == lib.E_ARG


def test_ch_scheme_checked_on_host(lib):
    g, w, p = _args(lib)
    p[0].ch_scheme = 7                                   # unknown scheme
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g, w, p)
    assert ei.value.status == lib.E_ARG
    ga, wa, pa = _args(lib)
    gb, wb, pb = _args(lib)
    pb[0].ch_scheme = lib.CH_EXPLICIT                    # one scheme per context
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(ga + gb, wa + wb, pa + pb)
    assert ei.value.status == lib.E_ARG


def test_tuning_calls_reject_a_null_context(lib):
    so = lib.lib()
    t = lib.Tuning()
    assert so.ib_pf_set_tuning(None, 0, ct.byref(t)) == lib.E_ARG
    assert so.ib_pf_get_tuning(None, 0, ct.byref(t)) == lib.E_ARG
    assert so.ib_pf_autotune(None, 0, 1, ct.byref(t), None) == lib.E_ARG


def test_split_bf16_form_limits_checked_on_host(lib):
    # the tensor-core z solve (FP32_3XBF16) is built for 3D grids with nz = 128 or 256
    g, w, p = _args(lib)
    p[0].precision = lib.FP32_3XBF16                     # 2D context
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g, w, p)
    assert ei.value.status == lib.E_UNSUPPORTED
    g, w, p = _args3(lib, n=(32, 32, 64), L=(1.0, 1.0, 2.0))
    p[0].precision = lib.FP32_3XBF16                     # nz = 64
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g, w, p)
    assert ei.value.status == lib.E_UNSUPPORTED
    g, w, p = _args3(lib)
    p[0].precision = 3                                   # unknown precision
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g, w, p)
    assert ei.value.status == lib.E_ARG


def test_mask_fractions_checked_on_host(lib):
    import numpy as np
    g, w, p = _args(lib)
    w[0] = lib.make_geometry(lib.WALL_MASK, [])                       # no fractions
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g, w, p)
    assert ei.value.status == lib.E_ARG
    nx, ny = 128, 64
    bad = [np.ones((ny, nx)), np.ones((ny, nx)), np.ones((ny + 1, nx))]
    bad[1][3, 5] = 1.5                                                # out of [0, 1]
    w[0] = lib.make_geometry(lib.WALL_MASK, [], alpha=bad)
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g, w, p)
    assert ei.value.status == lib.E_ARG
    assert "MASK" in lib.ib_pf_last_error(None)
    g3, w3, p3 = _args3(lib)
    n = 32
    bad3 = [np.ones((n, n, n))] * 3 + [np.ones((n + 1, n, n))]
    bad3[3] = bad3[3].copy()
    bad3[3][0, 0, 0] = np.nan                                         # not finite
    w3[0] = lib.make_geometry(lib.WALL_MASK, [], alpha=bad3)
    with pytest.raises(lib.IbPfError) as ei:
        lib.ib_pf_init_geometry(g3, w3, p3)
    assert ei.value.status == lib.E_ARG
