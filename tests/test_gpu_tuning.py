"""The autotuner's launch shapes change how cells are grouped into work, never a
cell's arithmetic: every compiled shape of every kernel family gives bitwise
the result of the default launch; a tuned choice is cached, reported, saved and
loaded; batch plans tune their CTA count and take the cached planes per work
item of the generic kernel."""
import math

import pytest
import torch

from gpu_helpers import random_case
from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(autouse=True)
def empty_cache():
    sl.sl_tuning_clear()
    yield
    sl.sl_tuning_clear()


def smooth(shape, dtype=torch.float32):
    nz, ny, nx = shape
    phi = W.random_modes(shape, W.draw_modes(3, 8, 3, seed=sum(shape)), dtype=dtype).to(DEV)
    vel = W.abc_velocity(shape, dtype=dtype).to(DEV)
    sp = [2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz]
    return phi, vel, sp, 0.45 * min(sp)


def step(phi, vel, sp, dt, scheme, parity, dtype="f32"):
    out = sl.advect(phi, vel, dt, sp, scheme, parity, delta64=(dtype == "f32_d64"))
    torch.cuda.synchronize()
    assert sl.sl_device_status() == 0
    return out


# (torch shape, scheme, dtype, kernel, [(tile_y, tile_z, ctas_per_sm), ...])
FORCED = [
    ((64, 64, 64), "CEC", sl.F32, 1, [(32, 0, 1), (32, 0, 2)]),
    ((24, 36, 40), "CEC", sl.F32, 2, [(32, 8, 0), (32, 24, 0), (32, 5, 0)]),
    ((20, 48, 64), "CIR", sl.F32, 3, [(16, 8, 0), (32, 20, 0), (32, 3, 0)]),
    ((20, 48, 64), "FEC", sl.F32, 4, [(8, 8, 0), (16, 20, 0), (32, 7, 0)]),
    ((20, 48, 64), "BEC", sl.F32, 4, [(8, 0, 1), (16, 0, 3), (32, 0, 2)]),
    ((12, 20, 24), "BEC", sl.F64, 4, [(8, 0, 1), (8, 0, 2)]),
    ((12, 20, 24), "FEC", sl.F64, 4, [(8, 5, 0)]),
]


@pytest.mark.parametrize("shape,scheme,dtype,kernel,shapes", FORCED)
def test_every_launch_shape_gives_the_default_bits(tmp_path, shape, scheme, dtype, kernel, shapes):
    name = "f64" if dtype == sl.F64 else "f32"
    phi, vel, sp, dt = smooth(shape, torch.float64 if dtype == sl.F64 else torch.float32)
    dims = list(shape[::-1])
    for parity in ((0, 1) if scheme == "CEC" else (0,)):
        ref = step(phi, vel, sp, dt, scheme, parity, name)
        for ty, tz, ctas in shapes:
            p = tmp_path / "shape.txt"
            p.write_text(f"{dims[0]} {dims[1]} {dims[2]} {sl.SCHEMES[scheme]} {dtype} {kernel} 32 {ty} {tz} {ctas} 1\n")
            sl.sl_tuning_load(str(p))
            got = step(phi, vel, sp, dt, scheme, parity, name)
            assert torch.equal(got, ref), (scheme, shape, ty, tz, ctas, parity)
            sl.sl_tuning_clear()


@pytest.mark.parametrize("shape,scheme", [((64, 64, 64), "CEC"), ((24, 36, 40), "CEC"), ((20, 48, 64), "CIR"),
                                          ((20, 48, 64), "FEC"), ((20, 48, 64), "BEC")])
def test_tuned_choice_is_cached_used_and_persists(tmp_path, shape, scheme):
    phi, vel, sp, dt = smooth(shape)
    dims = list(shape[::-1])
    ref = step(phi, vel, sp, dt, scheme, 1)
    t = sl.sl_autotune_scheme(torch.empty_like(phi), phi, vel, 3, dims, sp, dt, sl.SCHEMES[scheme], sl.F32)
    assert t.kernel in (1, 2, 3, 4) and t.ms > 0 and t.tile_x == 32 and t.tile_y in (8, 16, 32)
    got = sl.sl_tuning_get(dims, sl.SCHEMES[scheme], sl.F32)
    assert got is not None and (got.kernel, got.tile_y, got.tile_z, got.ctas_per_sm) == \
        (t.kernel, t.tile_y, t.tile_z, t.ctas_per_sm)
    assert torch.equal(step(phi, vel, sp, dt, scheme, 1), ref)
    p = tmp_path / "tuned.txt"
    sl.sl_tuning_save(str(p))
    sl.sl_tuning_clear()
    assert sl.sl_tuning_get(dims, sl.SCHEMES[scheme], sl.F32) is None
    sl.sl_tuning_load(str(p))
    back = sl.sl_tuning_get(dims, sl.SCHEMES[scheme], sl.F32)
    assert (back.kernel, back.tile_y, back.tile_z, back.ctas_per_sm) == (t.kernel, t.tile_y, t.tile_z, t.ctas_per_sm)
    assert torch.equal(step(phi, vel, sp, dt, scheme, 1), ref)


def test_former_autotune_interface_keeps_results():
    phi, vel, sp, dt = random_case((40, 36, 44), seed=4)
    p, v = phi.to(DEV), vel.to(DEV)
    ref = step(p, v, sp, dt, "CEC", 0)
    tz = sl.sl_autotune(torch.empty_like(p), p, v, 3, [44, 36, 40], sp, dt, sl.F32)
    assert 1 <= tz <= 40
    assert sl.sl_tuning_get([44, 36, 40], sl.CEC, sl.F32).tile_z == tz
    assert torch.equal(step(p, v, sp, dt, "CEC", 0), ref)


def _instances(shapes):
    keep, recs = [], []
    for shape in shapes:
        phi, vel, sp, dt = smooth(shape)
        a, b = phi.clone(), torch.empty_like(phi)
        keep.append((a, b, vel))
        recs.append(sl.Instance(a.data_ptr(), b.data_ptr(), vel.data_ptr(), tuple(shape[::-1]), tuple(sp), dt))
    return keep, recs


@pytest.mark.parametrize("shapes,kernel", [([(64, 64, 64), (32, 96, 64), (40, 64, 128)], 1),
                                           ([(24, 36, 40), (64, 64, 64), (17, 20, 52)], 2)])
def test_batch_autotune_keeps_results(shapes, kernel):
    keep, recs = _instances(shapes)
    h = sl.sl_batch_create(recs)
    try:
        before = sl.sl_batch_tuning(h)
        assert before.kernel == kernel
        sl.sl_batch_step(h, 0)
        torch.cuda.synchronize()
        ref = [b.clone() for _, b, _ in keep]
        t = sl.sl_batch_autotune(h)
        assert t.kernel == kernel and t.ctas_per_sm >= 1 and t.ms > 0
        now = sl.sl_batch_tuning(h)
        assert (now.ctas_per_sm, now.ms) == (t.ctas_per_sm, t.ms)
        for _, b, _ in keep:
            b.zero_()
        sl.sl_batch_step(h, 0)
        torch.cuda.synchronize()
        for (_, b, _), r in zip(keep, ref):
            assert torch.equal(b, r)
        assert sl.sl_device_status() == 0
    finally:
        sl.sl_batch_destroy(h)


def test_batch_takes_the_cached_planes_per_item():
    shape = (24, 36, 40)   # served by the generic split kernel
    phi, vel, sp, dt = smooth(shape)
    t = sl.sl_autotune_scheme(torch.empty_like(phi), phi, vel, 3, list(shape[::-1]), sp, dt, sl.CEC, sl.F32)
    assert t.kernel == 2 and t.tile_z >= 1
    keep, recs = _instances([shape, (64, 64, 64)])
    h = sl.sl_batch_create(recs)
    try:
        assert sl.sl_batch_tuning(h).tile_z == t.tile_z
    finally:
        sl.sl_batch_destroy(h)
