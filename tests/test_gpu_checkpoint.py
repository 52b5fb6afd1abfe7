"""Checkpoints of fields and of the learned corrector: bitwise round trips, a
resumed run equal to an uninterrupted one, and files of another grid or type,
truncated or corrupted files refused without touching the device field."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import random_case
from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("dtype,tdt", [(sl.F32, torch.float32), (sl.F64, torch.float64), (sl.F32_D64, torch.float32)])
@pytest.mark.parametrize("shape", [(9, 10, 12), (1, 17, 23)])
def test_field_round_trip_is_bitwise(tmp_path, shape, dtype, tdt):
    ndim = 2 if shape[0] == 1 else 3
    dims = list(shape[::-1])
    f = torch.randn(shape, dtype=tdt, device=DEV)
    p = tmp_path / "f.slf"
    sl.sl_field_save(str(p), f, ndim, dims, dtype, step=123)
    g = torch.full_like(f, 7.0)
    assert sl.sl_field_load(str(p), g, ndim, dims, dtype) == 123
    assert torch.equal(f, g)
    header = p.read_bytes().split(b"\n", 1)[0].decode()
    assert '"format": "libsl-field"' in header and f'"step": 123' in header


def test_resumed_run_equals_the_uninterrupted_run(tmp_path):
    shape = (32, 32, 64)
    nz, ny, nx = shape
    phi = W.random_modes(shape, W.draw_modes(3, 8, 3, seed=1), device=DEV, dtype=torch.float32)
    vel = W.abc_velocity(shape, device=DEV, dtype=torch.float32)
    sp = [2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz]
    dt = 0.4 * min(sp)

    def run(cur, k0, k1):
        for k in range(k0, k1):
            cur = sl.advect(cur, vel, dt, sp, "CEC", k)
        return cur

    full = run(phi.clone(), 0, 10)
    half = run(phi.clone(), 0, 5)
    p = tmp_path / "state.slf"
    sl.sl_field_save(str(p), half, 3, [nx, ny, nz], sl.F32, step=5)
    back = torch.empty_like(half)
    k = sl.sl_field_load(str(p), back, 3, [nx, ny, nz], sl.F32)
    assert k == 5
    torch.cuda.synchronize()
    assert torch.equal(run(back, k, 10), full)


def _mangle(p, how):
    raw = bytearray(p.read_bytes())
    head = raw.index(b"\n") + 1
    if how == "flip":
        raw[head + 17] ^= 0x10
    elif how == "truncate":
        raw = raw[:-3]
    elif how == "trailing":
        raw += b"\0"
    elif how == "header":
        raw[2:8] = b"XXXXXX"
    p.write_bytes(bytes(raw))


@pytest.mark.parametrize("how", ["flip", "truncate", "trailing", "header"])
def test_damaged_field_file_is_refused(tmp_path, how):
    f = torch.randn((5, 6, 8), device=DEV)
    p = tmp_path / "f.slf"
    sl.sl_field_save(str(p), f, 3, [8, 6, 5], sl.F32)
    _mangle(p, how)
    g = torch.full_like(f, 3.0)
    with pytest.raises(sl.SLError) as e:
        sl.sl_field_load(str(p), g, 3, [8, 6, 5], sl.F32)
    assert e.value.code == -1
    assert torch.equal(g, torch.full_like(f, 3.0))


@pytest.mark.parametrize("dims,dtype", [([8, 6, 4], sl.F32), ([6, 8, 5], sl.F32), ([8, 6, 5], sl.F64)])
def test_file_of_another_grid_or_type_is_refused(tmp_path, dims, dtype):
    f = torch.randn((5, 6, 8), device=DEV)
    p = tmp_path / "f.slf"
    sl.sl_field_save(str(p), f, 3, [8, 6, 5], sl.F32)
    g = torch.zeros((dims[2], dims[1], dims[0]), dtype=torch.float64 if dtype == sl.F64 else torch.float32, device=DEV)
    with pytest.raises(sl.SLError) as e:
        sl.sl_field_load(str(p), g, 3, dims, dtype)
    assert e.value.code == -1
    assert not g.any()


def test_corrector_weights_round_trip(tmp_path):
    shape = (32, 32, 32)
    phi, vel, sp, dt = random_case(shape, seed=2, cmax=0.6)
    phi, vel = phi.to(DEV), vel.to(DEV)
    dims = list(shape[::-1])
    c = sl.sl_corrector_create(11)
    d = sl.sl_corrector_create(12)
    try:
        nxt = sl.advect(phi, vel, dt, sp, "CEC", 0)
        sl.sl_corrector_add_samples(c, phi, nxt, vel, dims, sp, dt, 20000, seed=1)
        sl.sl_corrector_train(c, 20, 1024, 1e-3, seed=2)
        p = tmp_path / "w.slc"
        sl.sl_corrector_save(c, str(p))
        sl.sl_corrector_load(d, str(p))
        assert np.array_equal(sl.sl_corrector_get_params(c), sl.sl_corrector_get_params(d))
        a, b = torch.empty_like(phi), torch.empty_like(phi)
        sl.sl_advect_learned(c, a, phi, vel, 3, dims, sp, dt, 0, check=0)
        sl.sl_advect_learned(d, b, phi, vel, 3, dims, sp, dt, 0, check=0)
        assert torch.equal(a, b)
        _mangle(p, "flip")
        before = sl.sl_corrector_get_params(d).copy()
        with pytest.raises(sl.SLError):
            sl.sl_corrector_load(d, str(p))
        assert np.array_equal(sl.sl_corrector_get_params(d), before)
    finally:
        sl.sl_corrector_destroy(c)
        sl.sl_corrector_destroy(d)
