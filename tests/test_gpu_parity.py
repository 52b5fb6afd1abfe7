"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: relative L2 <= 1e-5 for float32 fields, <= 1e-12 for float64 fields,
element-wise against the oracle on the same seeded inputs; sizes span several
tiles, z chunks and ragged tails; full-size grids are checked on sampled cells.
"""
import math
import zlib

import numpy as np
import pytest
import torch

from gpu_helpers import (TOL, TORCH_DT, assert_parity, courant, oracle_at_cells, oracle_step, random_case,
                         rel_l2, sample_cells)
from oracle import oracle as O
from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"

SHAPES_3D = [(5, 5, 5), (11, 9, 7), (37, 45, 68), (9, 10, 12), (3, 4, 40),
             (16, 32, 64), (9, 64, 96)]      # the last two take the bulk-copy CEC path in FP32
SHAPES_2D = [(13, 17), (40, 64), (1, 8)]
SCHEMES = ["CIR", "FEC", "BEC", "CEC"]


def gpu_step(phi, vel, spacing, dt, scheme, parity, dtype):
    return sl.advect(phi.to(DEV), vel.to(DEV), dt, spacing, scheme, parity, delta64=(dtype == "f32_d64"))


@pytest.mark.parametrize("dtype", ["f32", "f64", "f32_d64"])
@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("shape", SHAPES_3D + SHAPES_2D)
def test_one_step_matches_oracle(shape, scheme, dtype):
    phi, vel, sp, dt = random_case(shape, seed=zlib.crc32(repr((shape, scheme)).encode()) % 1000, dtype=dtype)
    for parity in ((0, 1) if scheme == "CEC" else (0,)):
        out = gpu_step(phi, vel, sp, dt, scheme, parity, dtype)
        torch.cuda.synchronize()
        ref = oracle_step(phi, vel, sp, dt, scheme, parity)
        assert_parity(out.cpu().numpy(), ref, dtype, f"{scheme} {dtype} {shape} parity {parity}")
    assert sl.sl_device_status() == 0


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_many_steps_smooth_flow(scheme, dtype):
    """20 steps of an ABC flow on a random-mode field (sweep order alternating)."""
    shape = (24, 28, 36)
    t = TORCH_DT[dtype]
    phi = W.random_modes(shape, W.draw_modes(3, 16, 4, seed=2), dtype=t)
    vel = W.abc_velocity(shape, dtype=t)
    sp = [2 * math.pi / n for n in shape[::-1]]
    dt = 0.8 * min(sp) / 2.0
    ref = phi.double().numpy()
    cur = phi.to(DEV)
    v = vel.to(DEV)
    c = courant(vel, sp, dt)
    for k in range(20):
        cur = sl.advect(cur, v, dt, sp, scheme, k)
        ref = O.step(ref, c, O.SCHEMES[scheme], k)
    assert_parity(cur.cpu().numpy(), ref, dtype, f"{scheme} {dtype} 20 steps", allowance=4)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_constant_field_is_preserved_bitwise(scheme, dtype):
    shape = (10, 12, 16)
    _, vel, sp, dt = random_case(shape, seed=3, dtype=dtype)
    phi = torch.full(shape, 1.625, dtype=TORCH_DT[dtype])
    for parity in (0, 1):
        out = gpu_step(phi, vel, sp, dt, scheme, parity, dtype).cpu()
        assert torch.equal(out, phi)


@pytest.mark.parametrize("dtype", ["f32", "f64", "f32_d64"])
@pytest.mark.parametrize("shape", [(8, 12, 16), (16, 32, 64)])   # generic kernels; the persistent CEC kernel
@pytest.mark.parametrize("scheme", SCHEMES)
def test_integer_courant_is_a_shift(scheme, shape, dtype):
    """Pin P2: Courant numbers of +-1 on every axis (and 0 on one) give the exact
    cyclic shift, bit for bit, in every scheme and both sweep orders."""
    rng = np.random.default_rng(4)
    t = TORCH_DT[dtype]
    phi = torch.from_numpy(rng.standard_normal(shape)).to(t)
    sp, dt = [1.0, 1.0, 1.0], 1.0
    for c, shifts in (((1.0, -1.0, 1.0), (1, -1, 1)), ((-1.0, 0.0, -1.0), (-1, 0, -1))):
        vel = torch.stack([torch.full(shape, v) for v in c]).to(t)
        for parity in ((0, 1) if scheme == "CEC" else (0,)):
            out = gpu_step(phi, vel, sp, dt, scheme, parity, dtype).cpu()
            assert torch.equal(out, torch.roll(phi, shifts=shifts, dims=(0, 1, 2))), (c, parity)


def test_courant_violation_sets_status_bit():
    shape = (8, 8, 8)
    phi, vel, sp, dt = random_case(shape, seed=5, cmax=0.5)
    vel[0, 3, 4, 5] = 1.5 * sp[0] / dt
    sl.sl_device_status()   # clear
    out = gpu_step(phi, vel, sp, dt, "CEC", 0, "f32")
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    assert sl.sl_device_status() & sl.DEV_CFL
    assert sl.sl_device_status() == 0   # read clears


def test_argument_errors():
    shape = (8, 8, 8)
    phi, vel, sp, dt = random_case(shape, seed=6)
    p, v = phi.to(DEV), vel.to(DEV)
    dims = [8, 8, 8]
    with pytest.raises(sl.SLError) as e:
        sl.sl_advect(p, p, v, 3, dims, sp, dt, sl.CEC, sl.F32)
    assert e.value.code == -2
    with pytest.raises(sl.SLError) as e:
        sl.sl_advect(torch.empty_like(p), p, v, 4, dims, sp, dt, sl.CEC, sl.F32)
    assert e.value.code == -1
    with pytest.raises(sl.SLError) as e:
        sl.sl_advect(torch.empty_like(p), p, v, 3, [8, 0, 8], sp, dt, sl.CEC, sl.F32)
    assert e.value.code == -1
    with pytest.raises(sl.SLError) as e:
        sl.sl_advect(torch.empty_like(p), p, v, 3, dims, sp, dt, 7, sl.F32)
    assert e.value.code == -1
    with pytest.raises(sl.SLError) as e:
        sl.sl_advect(torch.empty_like(p), p, v, 3, dims, [0.1, -1.0, 0.1], dt, sl.CEC, sl.F32)
    assert e.value.code == -1
    with pytest.raises(sl.SLError) as e:
        sl.sl_advect(v[0], p, v, 3, dims, sp, dt, sl.CEC, sl.F32)
    assert e.value.code == -2


def test_unaligned_pointers_use_the_scalar_staging():
    shape = (6, 8, 12)
    phi, vel, sp, dt = random_case(shape, seed=7)
    n = phi.numel()
    buf = torch.empty(n + 1, device=DEV)
    buf[1:] = phi.to(DEV).reshape(-1)
    out = torch.empty(n + 1, device=DEV)
    sl.sl_advect(out[1:], buf[1:], vel.to(DEV), 3, [12, 8, 6], sp, dt, sl.CEC, sl.F32, 0)
    torch.cuda.synchronize()
    ref = oracle_step(phi, vel, sp, dt, "CEC", 0)
    assert_parity(out[1:].reshape(shape).cpu().numpy(), ref, "f32", "misaligned buffers")


def test_multi_field_equals_single_calls():
    shape = (12, 16, 20)
    _, vel, sp, dt = random_case(shape, seed=8)
    v = vel.to(DEV)
    fields = [torch.randn(shape, device=DEV) for _ in range(4)]
    outs = [torch.empty_like(f) for f in fields]
    sl.sl_advect_multi(outs, fields, v, 3, [20, 16, 12], sp, dt, sl.CEC, sl.F32, 1)
    for f, o in zip(fields, outs):
        assert torch.equal(o, sl.advect(f, v, dt, sp, "CEC", 1))


@pytest.mark.parametrize("nfields", [1, 2, 3, 4, 6])
@pytest.mark.parametrize("parity", [0, 1])
def test_multi_field_launch_equals_single_calls(nfields, parity):
    """On the persistent kernel's geometry one launch advances up to four fields
    (groups of CTAs share the velocity reads); six fields take two launches.
    Every field equals its single-field step bit for bit, and the first matches
    the oracle cell by cell."""
    shape = (40, 64, 96)
    _, vel, sp, dt = random_case(shape, seed=90 + nfields, cmax=0.9)
    v = vel.to(DEV)
    fields = [torch.randn(shape, device=DEV) for _ in range(nfields)]
    outs = [torch.empty_like(f) for f in fields]
    sl.sl_device_status()
    sl.sl_advect_multi(outs, fields, v, 3, [96, 64, 40], sp, dt, sl.CEC, sl.F32, parity)
    torch.cuda.synchronize()
    assert sl.sl_device_status() == 0
    for f, o in zip(fields, outs):
        assert torch.equal(o, sl.advect(f, v, dt, sp, "CEC", parity))
    assert_parity(outs[0].cpu().numpy(), oracle_step(fields[0].cpu(), vel, sp, dt, "CEC", parity), "f32",
                  f"multi-field {nfields} parity {parity}")


@pytest.mark.parametrize("dtype", ["f32", "f64", "f32_d64"])
@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("shape", [(6, 20, 36), (1, 42, 56), (8, 16, 64)])
def test_strided_fields_share_one_launch_and_equal_single_calls(shape, scheme, dtype):
    """Fields stored back to back (uniform strides, one alignment) go through
    the generic kernels in one launch with a field index per CTA row (the
    four-cell CIR kernel, which (8, 16, 64) in FP32 reaches, takes them one
    launch each); every field equals its single-field step bit for bit, the
    first matches the oracle.  Fields at an odd FP32 plane size have mixed 16-byte alignment and
    take one launch each; the results are the same."""
    nd = 2 if shape[0] == 1 else 3
    shp = shape[1:] if nd == 2 else shape
    phi, vel, sp, dt = random_case(shp, seed=sum(shp) + len(scheme), dtype=dtype)
    t = TORCH_DT[dtype]
    v = vel.to(DEV)
    dims = list(shp[::-1]) + ([1] if nd == 2 else [])
    d64 = dtype == "f32_d64"
    code = {"f32": sl.F32, "f64": sl.F64, "f32_d64": sl.F32_D64}[dtype]
    for extra in (0, 1):   # extra = 1: an odd element between planes
        n = phi.numel()
        ins = torch.randn(3 * (n + extra), dtype=t, device=DEV)
        outs = torch.zeros(3 * (n + extra), dtype=t, device=DEV)
        fi = [ins[f * (n + extra):f * (n + extra) + n].view(shp) for f in range(3)]
        fo = [outs[f * (n + extra):f * (n + extra) + n].view(shp) for f in range(3)]
        for parity in ((0, 1) if scheme == "CEC" else (0,)):
            sl.sl_device_status()
            sl.sl_advect_multi(fo, fi, v, nd, dims, sp, dt, sl.SCHEMES[scheme], code, parity)
            torch.cuda.synchronize()
            assert sl.sl_device_status() == 0
            for a, b in zip(fi, fo):
                assert torch.equal(b, sl.advect(a.contiguous(), v, dt, sp, scheme, parity, delta64=d64)), (extra, parity)
        assert_parity(fo[0].cpu().numpy(), oracle_step(fi[0].cpu(), vel, sp, dt, scheme, parity), dtype,
                      f"strided {scheme} {dtype} {shape}")


def test_host_buffers_equal_device_path():
    shape = (16, 20, 24)
    phi, vel, sp, dt = random_case(shape, seed=9)
    out = torch.empty_like(phi).pin_memory()
    sl.sl_advect_host(out, phi.pin_memory(), vel.pin_memory(), 3, [24, 20, 16], sp, dt, sl.BEC, sl.F32, 0)
    assert torch.equal(out, sl.advect(phi.to(DEV), vel.to(DEV), dt, sp, "BEC", 0).cpu())


@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("shape", [(64, 32, 64), (96, 64, 64), (263, 32, 64), (40, 32, 64)])
def test_host_buffers_in_z_slabs_equal_device_path(shape, parity):
    """A CEC step on host buffers over the fast geometry runs in z slabs (2, 3
    and 8 slabs, the last with slabs of 32 and 33 planes; nz = 40 runs in one
    piece).  Each slab reads the input planes its halo reaches across slab
    edges and across the periodic boundary.  A step on other inputs of the same
    shape runs first, so a plane copied late or not at all leaves a stale value
    in the device staging buffer.  The result equals the device-buffer step
    bit for bit."""
    phi, vel, sp, dt = random_case(shape, seed=70 + shape[0], cmax=0.9)
    dims = [shape[2], shape[1], shape[0]]
    other = torch.randn(shape).pin_memory()
    junk = torch.empty(shape).pin_memory()
    sl.sl_advect_host(junk, other, (vel.flip(1) * 0.5).contiguous().pin_memory(), 3, dims, sp, dt,
                      sl.CEC, sl.F32, parity)
    out = torch.empty(shape).pin_memory()
    sl.sl_device_status()
    sl.sl_advect_host(out, phi.pin_memory(), vel.pin_memory(), 3, dims, sp, dt, sl.CEC, sl.F32, parity)
    assert sl.sl_device_status() == 0
    assert torch.equal(out, sl.advect(phi.to(DEV), vel.to(DEV), dt, sp, "CEC", parity).cpu())
    if shape[0] == 96 and parity == 0:
        assert_parity(out.numpy(), oracle_step(phi, vel, sp, dt, "CEC", 0), "f32", "z slabs")


def test_host_buffers_in_z_slabs_from_pageable_memory():
    """Pageable (not page-locked) host buffers take the same slab path; the
    copies are then staged by the driver, the result is the same."""
    shape = (96, 32, 64)
    phi, vel, sp, dt = random_case(shape, seed=82, cmax=0.9)
    dims = [shape[2], shape[1], shape[0]]
    out = torch.empty(shape)
    for parity in (0, 1):
        sl.sl_advect_host(out, phi, vel, 3, dims, sp, dt, sl.CEC, sl.F32, parity)
        assert torch.equal(out, sl.advect(phi.to(DEV), vel.to(DEV), dt, sp, "CEC", parity).cpu())


def test_host_buffers_in_z_slabs_flag_courant_violations():
    """A violation in any slab, including the cells next to slab edges, sets
    the status bit of a host-buffer step."""
    shape = (96, 32, 64)
    phi, vel, sp, dt = random_case(shape, seed=81, cmax=0.5)
    dims = [shape[2], shape[1], shape[0]]
    out = torch.empty(shape).pin_memory()
    for z in (0, 31, 32, 95):
        v = vel.clone()
        v[2, z, 5, 7] = 1.5 * sp[2] / dt
        sl.sl_device_status()
        sl.sl_advect_host(out, phi.pin_memory(), v.pin_memory(), 3, dims, sp, dt, sl.CEC, sl.F32, z & 1)
        assert sl.sl_device_status() & sl.DEV_CFL, z


@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_fast_path_courant_violation_each_axis(axis, parity):
    """The fused fast kernels flag |C| > 1 on any axis, at interior and seam cells."""
    shape = (16, 64, 64)                       # (nz, ny, nx): takes the fast path
    phi, vel, sp, dt = random_case(shape, seed=11, cmax=0.5)
    sl.sl_device_status()
    gpu_step(phi, vel, sp, dt, "CEC", parity, "f32")
    torch.cuda.synchronize()
    assert sl.sl_device_status() == 0
    for (z, y, x) in [(5, 20, 37), (0, 0, 0), (15, 63, 63), (7, 31, 32)]:
        v = vel.clone()
        v[axis, z, y, x] = -1.5 * sp[axis] / dt
        gpu_step(phi, v, sp, dt, "CEC", parity, "f32")
        torch.cuda.synchronize()
        assert sl.sl_device_status() & sl.DEV_CFL, (axis, parity, z, y, x)
        assert sl.sl_device_status() == 0


def test_norms_and_courant_reductions():
    shape = (30, 40, 50)
    a = torch.randn(shape, dtype=torch.float64, device=DEV)
    b = torch.randn(shape, dtype=torch.float64, device=DEV)
    got = sl.sl_norms(a, b, a.numel(), sl.F64)
    ref = O.norms(a.cpu().numpy(), b.cpu().numpy())
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    phi, vel, sp, dt = random_case(shape, seed=10, cmax=0.7)
    cmax = sl.sl_courant_max(vel.to(DEV), 3, [50, 40, 30], sp, dt, sl.F32)
    assert cmax == pytest.approx(np.abs(courant(vel, sp, dt)).max(), rel=1e-15)


@pytest.mark.parametrize("shape,parity", [((256, 256, 256), 0), ((256, 256, 256), 1),
                                          ((512, 512, 512), 0), ((512, 512, 512), 1)])
def test_full_size_sampled_parity(shape, parity):
    """The benchmark workload (256^3 ABC flow, 32-mode field, CFL 0.8) at full size in
    the launch configuration the benchmark times, and the same flow at 512^3 (the
    size of the four-field run), checked on 1500 sampled cells."""
    sp = [2 * math.pi / n for n in shape[::-1]]
    dt = 0.8 * sp[0] / 2.0
    phi = W.random_modes(shape, W.draw_modes(3, 32, 8, seed=0), device=DEV, dtype=torch.float32)
    vel = W.abc_velocity(shape, device=DEV, dtype=torch.float32)
    out = sl.advect(phi, vel, dt, sp, "CEC", parity)
    cells = sample_cells(shape, 1500, seed=11 + parity)
    ref = oracle_at_cells(phi, vel, sp, dt, "CEC", parity, cells)
    got = out[cells[:, 2], cells[:, 1], cells[:, 0]].cpu().double().numpy()
    assert_parity(got, ref, "f32", f"{shape} parity {parity}, sampled cells")


@pytest.mark.parametrize("scheme", ["CIR", "FEC", "BEC"])
def test_full_size_unsplit_sampled_parity(scheme):
    """The unsplit kernels (one fused launch per CIR / FEC / BEC step) on the
    benchmark workload at full size (256^3 ABC flow, 32-mode field, CFL 0.8), in
    the launch configuration the benchmark times, against the oracle on 1500
    sampled cells (an unsplit BEC output reads Phi within 3 cells per axis)."""
    shape = (256, 256, 256)
    sp = [2 * math.pi / n for n in shape[::-1]]
    dt = 0.8 * sp[0] / 2.0
    phi = W.random_modes(shape, W.draw_modes(3, 32, 8, seed=0), device=DEV, dtype=torch.float32)
    vel = W.abc_velocity(shape, device=DEV, dtype=torch.float32)
    sl.sl_device_status()
    out = sl.advect(phi, vel, dt, sp, scheme, 0)
    torch.cuda.synchronize()
    assert sl.sl_device_status() == 0
    cells = sample_cells(shape, 1500, seed=17)
    ref = oracle_at_cells(phi, vel, sp, dt, scheme, 0, cells)
    got = out[cells[:, 2], cells[:, 1], cells[:, 0]].cpu().double().numpy()
    assert_parity(got, ref, "f32", f"{scheme} 256^3, sampled cells")


@pytest.mark.parametrize("parity", [0, 1])
def test_batch_of_48_uneven_grids_sampled_parity(parity):
    """The batched workload (48 grids of sizes drawn from {64, 96, 128, 160,
    192}^3, ABC or Taylor-Green velocity with amplitudes in [0.5, 1.5], 32-mode
    field, CFL 0.8), one step as the benchmark runs it (one persistent launch,
    replayed from a captured CUDA graph), against the oracle on 40 sampled cells
    of every grid."""
    insts = W.draw_batch(48, seed=0)
    recs, keep = [], []
    for inst in insts:
        phi, vel = W.instance_fields(inst, device=DEV, dtype=torch.float32)
        n = inst.n
        sp = [2 * math.pi / n] * 3
        dt = 0.8 * sp[0] / float(vel.abs().amax())
        a, b = phi, torch.empty_like(phi)
        keep.append((a, b, vel, n, sp, dt))
        recs.append(sl.Instance(a.data_ptr(), b.data_ptr(), vel.data_ptr(), (n, n, n), tuple(sp), dt))
    h = sl.sl_batch_create(recs)
    try:
        sl.sl_device_status()
        if parity == 1:          # an odd step reads the B buffers
            for a, b, *_ in keep:
                b.copy_(a)
        sl.sl_batch_step(h, parity)      # first launch outside capture (per-device setup)
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                sl.sl_batch_step(h, parity, side)
        torch.cuda.current_stream().wait_stream(side)
        g.replay()
        torch.cuda.synchronize()
        assert sl.sl_device_status() == 0
    finally:
        sl.sl_batch_destroy(h)
    for i, (a, b, vel, n, sp, dt) in enumerate(keep):
        src, dst = (a, b) if parity == 0 else (b, a)
        cells = sample_cells((n, n, n), 40, seed=100 + i)
        ref = oracle_at_cells(src, vel, sp, dt, "CEC", parity, cells)
        got = dst[cells[:, 2], cells[:, 1], cells[:, 0]].cpu().double().numpy()
        assert_parity(got, ref, "f32", f"grid {i} ({n}^3, {insts[i].flow}) parity {parity}")


def test_generic_batched_kernel_matches_the_oracle():
    """A batch whose grids are not all whole 32 x 32 column tiles runs the
    generic work-queue kernel; three steps of every grid against three oracle
    steps (alternating sweep order)."""
    sizes = [(64, 64, 64), (32, 96, 32), (40, 24, 48), (16, 16, 16), (33, 20, 52)]
    insts, keep = [], []
    for i, s in enumerate(sizes):
        sp = [2 * math.pi / n for n in s[::-1]]
        phi = W.random_modes(s, W.draw_modes(3, 8, 4, seed=i), device=DEV, dtype=torch.float32)
        vel = W.abc_velocity(s, A=1.0 + 0.1 * i, device=DEV, dtype=torch.float32)
        dt = 0.8 * min(sp) / 2.5
        a, b = phi.clone(), torch.empty_like(phi)
        keep.append((a, b, vel, sp, dt, phi))
        insts.append(sl.Instance(a.data_ptr(), b.data_ptr(), vel.data_ptr(), (s[2], s[1], s[0]), tuple(sp), dt))
    h = sl.sl_batch_create(insts, tile_z=16)
    try:
        for k in range(3):
            sl.sl_batch_step(h, k)
        torch.cuda.synchronize()
    finally:
        sl.sl_batch_destroy(h)
    for a, b, vel, sp, dt, phi in keep:
        ref = phi.double().cpu().numpy()
        c = courant(vel, sp, dt)
        for k in range(3):
            ref = O.step(ref, c, O.CEC, k)
        assert_parity(b.cpu().numpy(), ref, "f32", f"{tuple(phi.shape)}, 3 steps", allowance=3)


def test_batched_equals_single_instance_steps():
    sizes = [(64, 64, 64), (32, 96, 32), (40, 24, 48), (16, 16, 16)]
    insts, keep, refs = [], [], []
    for i, s in enumerate(sizes):
        sp = [2 * math.pi / n for n in s[::-1]]
        phi = W.random_modes(s, W.draw_modes(3, 8, 4, seed=i), device=DEV, dtype=torch.float32)
        vel = W.abc_velocity(s, A=1.0 + 0.1 * i, device=DEV, dtype=torch.float32)
        dt = 0.8 * min(sp) / 2.5
        a, b = phi.clone(), torch.empty_like(phi)
        keep.append((a, b, vel, sp, dt, phi))
        insts.append(sl.Instance(a.data_ptr(), b.data_ptr(), vel.data_ptr(), (s[2], s[1], s[0]),
                                 tuple(sp), dt))
    h = sl.sl_batch_create(insts, tile_z=16)
    try:
        for k in range(3):
            sl.sl_batch_step(h, k)
        torch.cuda.synchronize()
    finally:
        sl.sl_batch_destroy(h)
    for a, b, vel, sp, dt, phi in keep:
        cur = phi
        for k in range(3):
            cur = sl.advect(cur, vel, dt, sp, "CEC", k)
        result = b if 3 % 2 == 1 else a
        # this mixed batch runs the generic kernel; a single 64^3 grid takes the
        # fast persistent kernel, whose float arithmetic is arranged differently
        assert rel_l2(result.cpu().double().numpy(), cur.cpu().double().numpy()) <= 1e-6


def test_autotune_keeps_results():
    shape = (64, 64, 64)
    phi, vel, sp, dt = random_case(shape, seed=12)
    p, v = phi.to(DEV), vel.to(DEV)
    before = sl.advect(p, v, dt, sp, "CEC", 0)
    choice = sl.sl_autotune(torch.empty_like(p), p, v, 3, [64, 64, 64], sp, dt, sl.F32)
    assert choice >= 1
    assert torch.equal(sl.advect(p, v, dt, sp, "CEC", 0), before)


@pytest.mark.parametrize("parity", [0, 1])
def test_fast_path_partitions_agree(parity):
    """The persistent CEC kernel splits (column tile, plane) pairs into equal
    shares; the same grid stepped alone and inside a batch with other grids
    (different shares and segment cuts) gives bitwise equal results, and both
    match the oracle."""
    shapes = [(24, 64, 96), (40, 32, 64), (8, 96, 64)]
    insts, keep = [], []
    for i, s in enumerate(shapes):
        phi, vel, sp, dt = random_case(s, seed=40 + i, spacing=[0.3, 0.2, 0.25])
        a, b = phi.to(DEV), torch.empty(s, device=DEV)
        v = vel.to(DEV)
        keep.append((phi, vel, a, b, v, sp, dt))
        insts.append(sl.Instance(a.data_ptr(), b.data_ptr(), v.data_ptr(), (s[2], s[1], s[0]), tuple(sp), dt))
    h = sl.sl_batch_create(insts)
    try:
        sl.sl_batch_step(h, parity)          # even: a -> b, odd: b -> a
        torch.cuda.synchronize()
    finally:
        sl.sl_batch_destroy(h)
    for phi, vel, a, b, v, sp, dt in keep:
        src, dst = (a, b) if parity == 0 else (b, a)
        single = sl.advect(src, v, dt, sp, "CEC", parity)
        assert torch.equal(dst, single)
        if parity == 0:
            ref = oracle_step(phi, vel, sp, dt, "CEC", 0)
            assert_parity(single.cpu().numpy(), ref, "f32", f"{tuple(phi.shape)}")


@pytest.mark.parametrize("parity", [0, 1])
def test_deformation_512_sampled_parity(parity):
    """The 512^3 time-reversing deformation flow of the four-field run: one
    multi-field step at t = 0 of the three velocity components and the
    random-mode scalar (one launch for the four fields), every field against
    the oracle on sampled cells."""
    n = 512
    shape = (n, n, n)
    vel = W.deformation_velocity(shape, device=DEV, dtype=torch.float32)
    sp = [1.0 / n] * 3
    dt = 0.8 * sp[0] / float(vel.abs().amax())
    scal = W.random_modes(shape, W.draw_modes(3, 32, 8, seed=5), length=1.0, device=DEV, dtype=torch.float32)
    ins = [vel[0].clone(), vel[1].clone(), vel[2].clone(), scal]
    outs = [torch.empty_like(f) for f in ins]
    sl.sl_advect_multi(outs, ins, vel, 3, [n, n, n], sp, dt, sl.CEC, sl.F32, parity)
    torch.cuda.synchronize()
    cells = sample_cells(shape, 600, seed=21 + parity)
    for f, o in zip(ins, outs):
        ref = oracle_at_cells(f, vel, sp, dt, "CEC", parity, cells)
        got = o[cells[:, 2], cells[:, 1], cells[:, 0]].cpu().double().numpy()
        assert_parity(got, ref, "f32", f"deformation field, parity {parity}")


def test_bounded_wait_times_out_and_reports():
    """A device wait that nothing completes gives up, sets SL_DEV_TIMEOUT and leaves
    the context usable (no fault, trap or hang)."""
    sl.sl_device_status()
    assert sl.sl_selftest_wait_timeout(2000) == -5
    assert sl.sl_device_status() & sl.DEV_TIMEOUT
    assert sl.sl_device_status() == 0
    x = torch.ones(4, device=DEV)
    assert float((x * 2).sum()) == 8.0
