"""The 3D schedule choices and the autotuner (ib_pf_set_tuning / ib_pf_autotune): every
choice gives the same step bit for bit, the tuner leaves the state as it found it, invalid
choices are refused, and the Python binding's JSON cache is keyed by shape, precision and
GPU."""
import json

import numpy as np
import pytest

from workloads import cases as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibpf():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf as m
    return m


def _case():
    # y and z axes of 256 points: both tile row widths are built for them
    return W.flat_wall_case3d(nx=16, ny=256, nz=256, wall_z=0.37 * 16 * (2.0 / 16), l_s=0.01)


def _solver(ibpf, prec):
    s = ibpf.solver_from_cases([_case()], prec)
    s.precompute_weights()
    s.write_state(W.random_state3d(_case(), seed=11))
    return s


def _snapshot(s):
    return {k: np.array(v, copy=True) for k, v in s.read_checkpoint().items()}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_choice_gives_the_same_steps(ibpf, prec):
    p = ibpf.FP64 if prec == "fp64" else ibpf.FP32
    out = []
    for choice in ({}, dict(y_tile_bytes=64, z_tile_bytes=64, predict_planes=8),
                   dict(y_tile_bytes=128, z_tile_bytes=128, predict_planes=32)):
        s = _solver(ibpf, p)
        s.set_tuning(0, **choice)
        s.step(3)
        assert s.query(ibpf.Q_STATUS) == 0.0
        out.append(_snapshot(s))
        s.close()
    for other in out[1:]:
        for k in out[0]:
            assert np.array_equal(out[0][k], other[k]), k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_keeps_the_state_and_sets_a_valid_choice(ibpf, prec):
    p = ibpf.FP64 if prec == "fp64" else ibpf.FP32
    s = _solver(ibpf, p)
    s.step(2)
    before = _snapshot(s)
    t, ms = ibpf.ib_pf_autotune(s.ctx, 0, 2)
    after = _snapshot(s)
    for k in before:
        assert np.array_equal(before[k], after[k]), k
    got = s.tuning(0)
    assert got == t.as_dict()
    assert got["y_tile_bytes"] in (64, 128) and got["z_tile_bytes"] in (64, 128)
    assert got["predict_planes"] in (8, 16, 32)
    assert all(ms[k] > 0 for k in ("y128", "y64", "z128", "z64", "planes8", "planes16", "planes32"))
    s.step(1)
    assert s.query(ibpf.Q_STATUS) == 0.0
    s.close()


def test_invalid_choices_are_refused(ibpf):
    s = _solver(ibpf, ibpf.FP32)
    for bad in (dict(y_tile_bytes=96), dict(z_tile_bytes=32), dict(predict_planes=12)):
        with pytest.raises(ibpf.IbPfError) as e:
            s.set_tuning(0, **bad)
        assert e.value.status == ibpf.E_ARG
    s.close()
    # 1024-point axes have no 128-byte tiles; 2D contexts have nothing to tune
    big = W.flat_wall_case3d(nx=16, ny=16, nz=1024, wall_z=0.37 * 16 * (2.0 / 16), l_s=0.01)
    s = ibpf.solver_from_cases([big], ibpf.FP32)
    with pytest.raises(ibpf.IbPfError) as e:
        s.set_tuning(0, z_tile_bytes=128)
    assert e.value.status == ibpf.E_ARG
    s.close()
    s2 = ibpf.solver_from_cases([W.flat_wall_128x64()], ibpf.FP32)
    with pytest.raises(ibpf.IbPfError) as e:
        s2.set_tuning(0, predict_planes=8)
    assert e.value.status == ibpf.E_UNSUPPORTED
    s2.close()


def test_json_cache_keyed_by_shape_precision_gpu(ibpf, tmp_path):
    cache = tmp_path / "tuning.json"
    s = _solver(ibpf, ibpf.FP32)
    first = s.autotune(0, reps=2, cache=cache, gpu_name="gpu-a")
    assert not first["cached"]
    table = json.loads(cache.read_text())
    assert list(table) == ["16x256x256:fp32:gpu-a"]
    s.close()
    s = _solver(ibpf, ibpf.FP32)
    again = s.autotune(0, reps=2, cache=cache, gpu_name="gpu-a")
    assert again["cached"] and again["choice"] == first["choice"]
    assert s.tuning(0) == first["choice"]
    other = s.autotune(0, reps=2, cache=cache, gpu_name="gpu-b")
    assert not other["cached"]
    assert sorted(json.loads(cache.read_text())) == ["16x256x256:fp32:gpu-a", "16x256x256:fp32:gpu-b"]
    s.close()
