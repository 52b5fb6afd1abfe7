"""Steps at any Courant number through the CUDA path (sl_advect_wide): parity
with the oracle's non-local schemes (CIR / FEC / BEC unsplit, CEC split with
the departure-cell correction, the oracle's CEC_SL), element by element on
seeded inputs with per-cell random Courant numbers up to 4.2, and the
properties that hold at any size: exact shifts, constants, agreement with the
local step below CFL 1, the cubic Lagrange interpolation at the departure point
for constant velocity, and the third order at CFL 3.75."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import TOL, assert_parity, rel_l2
from oracle import oracle as O
from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
ORACLE = {"CIR": O.CIR, "FEC": O.FEC, "BEC": O.BEC, "CEC": O.CEC_SL}
TORCH = {"f32": torch.float32, "f64": torch.float64}
NP = {"f32": np.float32, "f64": np.float64}


def case(shape, cmax, seed, dtype):
    """Field, velocity (CUDA tensors of dtype), spacing, dt and the Courant
    numbers exactly as the kernels form them (u_d times dt/dx_d rounded in dtype)."""
    nd = len(shape)
    rng = np.random.default_rng(seed)
    sp = [0.5, 0.25, 2.0][:nd]
    dt = 0.1
    phi = rng.standard_normal(shape)
    C = rng.uniform(-cmax, cmax, size=(nd,) + shape)
    vel = np.stack([C[d] * sp[d] / dt for d in range(nd)]).astype(NP[dtype])
    s = [NP[dtype](dt / sp[d]) for d in range(nd)]
    courant = np.stack([(vel[d] * s[d]).astype(np.float64) for d in range(nd)])
    return (torch.from_numpy(phi).to(TORCH[dtype]).to(DEV), torch.from_numpy(vel).to(DEV), sp, dt, courant)


def oracle_of(phi, courant, scheme, parity):
    return O.step(phi.double().cpu().numpy(), courant, ORACLE[scheme], parity)


# the last two have lines along x too long for the fused shared-memory sweep
# (FP64 beyond 4096 cells, FP32 beyond 8192), so their x sweep takes the three gathers
SHAPES = [(12, 10, 16), (9, 20, 24), (5, 7, 33), (40, 56), (17, 3), (6, 4100), (3, 8200)]


@pytest.mark.parametrize("cmax", [0.9, 2.5, 4.2])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["CIR", "FEC", "BEC", "CEC"])
@pytest.mark.parametrize("shape", SHAPES)
def test_one_step_matches_the_oracle(shape, scheme, dtype, cmax):
    phi, vel, sp, dt, courant = case(shape, cmax, 50 + len(shape) + int(10 * cmax), dtype)
    for parity in ((0, 1) if scheme == "CEC" else (0,)):
        sl.sl_device_status()
        got = sl.advect_wide(phi, vel, dt, sp, scheme, parity)
        torch.cuda.synchronize()
        assert sl.sl_device_status() == 0
        assert_parity(got.cpu().numpy(), oracle_of(phi, courant, scheme, parity), dtype,
                      f"{scheme} {dtype} {shape} cmax {cmax} parity {parity}")


@pytest.mark.parametrize("scheme", ["CIR", "FEC", "BEC", "CEC"])
def test_integer_courant_is_an_exact_shift(scheme):
    shape = (6, 7, 9)
    phi = torch.randn(shape, device=DEV)
    vel = torch.stack([torch.full(shape, v, device=DEV) for v in (3.0, -2.0, 1.0)])
    got = sl.advect_wide(phi, vel, 1.0, [1.0, 1.0, 1.0], scheme, 0)
    assert torch.equal(got, torch.roll(phi, shifts=(1, -2, 3), dims=(0, 1, 2)))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["CIR", "FEC", "BEC", "CEC"])
def test_constant_field_is_preserved_bitwise(scheme, dtype):
    shape = (10, 12, 16)
    _, vel, sp, dt, _ = case(shape, 3.3, 61, dtype)
    phi = torch.full(shape, 1.625, dtype=TORCH[dtype], device=DEV)
    for parity in (0, 1):
        assert torch.equal(sl.advect_wide(phi, vel, dt, sp, scheme, parity), phi)


@pytest.mark.parametrize("scheme", ["CIR", "FEC", "BEC", "CEC"])
def test_below_cfl_one_equals_the_local_step(scheme):
    shape = (12, 32, 64)
    phi, vel, sp, dt, _ = case(shape, 0.95, 62, "f64")
    for parity in (0, 1):
        wide = sl.advect_wide(phi, vel, dt, sp, scheme, parity)
        local = sl.advect(phi, vel, dt, sp, scheme, parity)
        assert rel_l2(wide.cpu().numpy(), local.cpu().numpy()) < 1e-13


def cubic_lagrange_at(line, X):
    n = len(line)
    b = np.floor(X).astype(np.int64)
    t = X - b
    nodes = [-1.0, 0.0, 1.0, 2.0]
    out = np.zeros_like(X)
    for k, xk in enumerate(nodes):
        w = np.ones_like(t)
        for xj in nodes:
            if xj != xk:
                w *= (t - xj) / (xk - xj)
        out += w * line[(b - 1 + k) % n]
    return out


@pytest.mark.parametrize("C", [1.3, 2.75, -3.6, 5.2])
def test_constant_velocity_cec_is_cubic_lagrange_at_the_departure_point(C):
    """The textbook 4-point interpolation at X = i - C along x (FP64; y, z at rest)."""
    shape = (8, 32, 37)
    rng = np.random.default_rng(63)
    line = rng.standard_normal(37)
    phi = torch.from_numpy(np.broadcast_to(line, shape).copy()).to(DEV)
    vel = torch.zeros((3,) + shape, dtype=torch.float64, device=DEV)
    vel[0] = C
    got = sl.advect_wide(phi, vel, 1.0, [1.0, 1.0, 1.0], "CEC", 0).cpu().numpy()
    want = cubic_lagrange_at(line, np.arange(37) - C)
    assert np.max(np.abs(got - want[None, None, :])) < 1e-13


def test_third_order_at_cfl_3_75():
    """Sec. 4: a Gaussian translated once around [0, 1) along z at CFL 3.75 (FP64):
    the CEC error falls by 2^3 per halving of dx, the literal reading's rate
    (2^2) would fail."""
    errs = []
    for n in (128, 256):
        shape = (n, 32, 64)
        g = W.gaussian((n,), [0.5], 0.1, images=2).double()
        phi0 = g.view(n, 1, 1).expand(shape).contiguous().to(DEV)
        dt, nsteps = W.dt_for_cfl(1.0, n, 3.75)
        vel = torch.zeros((3,) + shape, dtype=torch.float64, device=DEV)
        vel[2] = 1.0
        sp = [1.0 / 64, 1.0 / 32, 1.0 / n]
        ws = torch.empty(sl.sl_advect_wide_workspace(3, [64, 32, n], sl.CEC, sl.F64) + 256, dtype=torch.uint8,
                         device=DEV)
        phi, out = phi0.clone(), torch.empty_like(phi0)
        for k in range(nsteps):
            sl.advect_wide(phi, vel, dt, sp, "CEC", k & 1, out=out, workspace=ws)
            phi, out = out, phi
        errs.append(torch.sqrt(((phi - phi0) ** 2).mean()).item())
    assert 2.8 < math.log2(errs[0] / errs[1]) < 3.3, errs


def test_argument_errors():
    shape = (8, 8, 8)
    phi, vel, sp, dt, _ = case(shape, 2.0, 64, "f32")
    out = torch.empty_like(phi)
    dims = [8, 8, 8]
    need = sl.sl_advect_wide_workspace(3, dims, sl.CEC, sl.F32)
    assert need == 4 * 2048 and sl.sl_advect_wide_workspace(3, dims, sl.CIR, sl.F32) == 0
    ws = torch.empty(need + 256, dtype=torch.uint8, device=DEV)
    base = ws.data_ptr() + (-ws.data_ptr()) % 256
    with pytest.raises(sl.SLError, match="SL_ERR_ARG"):        # too small
        sl.sl_advect_wide(out, phi, vel, 3, dims, sp, dt, sl.CEC, sl.F32, 0, base, need - 1)
    with pytest.raises(sl.SLError, match="SL_ERR_ARG"):        # misaligned
        sl.sl_advect_wide(out, phi, vel, 3, dims, sp, dt, sl.CEC, sl.F32, 0, base + 4, need)
    with pytest.raises(sl.SLError, match="SL_ERR_ALIAS"):      # out is the input
        sl.sl_advect_wide(phi, phi, vel, 3, dims, sp, dt, sl.CEC, sl.F32, 0, base, need)
    with pytest.raises(sl.SLError, match="SL_ERR_ALIAS"):      # workspace holds the output
        sl.sl_advect_wide(base, phi, vel, 3, dims, sp, dt, sl.CEC, sl.F32, 0, base, need)
    with pytest.raises(sl.SLError, match="SL_ERR_UNSUPPORTED"):
        sl.sl_advect_wide(out, phi, vel, 3, dims, sp, dt, sl.CEC, sl.F32_D64, 0, base, need)
    sl.sl_advect_wide(out, phi, vel, 3, dims, sp, dt, sl.CEC, sl.F32, 0, base, need)
    torch.cuda.synchronize()


def test_non_finite_velocity_is_flagged_and_stays_in_bounds():
    shape = (8, 16, 16)
    phi, vel, sp, dt, _ = case(shape, 2.0, 65, "f32")
    vel[0, 3, 4, 5] = float("nan")
    vel[2, 1, 2, 3] = float("inf")
    sl.sl_device_status()
    for scheme in ("CIR", "CEC"):
        got = sl.advect_wide(phi, vel, dt, sp, scheme, 0)
        torch.cuda.synchronize()
        assert sl.sl_device_status() & sl.DEV_CFL
        assert got.shape == phi.shape


@pytest.mark.parametrize("parity", [0, 1])
def test_full_size_sampled_parity_at_cfl_3_64(parity):
    """The benchmark's large-CFL configuration (256^3 ABC flow, 32-mode field,
    CFL 3.64, the fused line sweeps) checked on 120 sampled cells.  A split CEC
    output reads Phi within 3 ceil(C) + 3 cells along each axis (L_U reaches
    ceil(C) + 1, delta another ceil(C) + 1, the correction ceil(C) + 1 more), so
    the oracle's step on the periodic window of radius 15 gives the full-grid
    value at its centre."""
    from gpu_helpers import sample_cells, windows
    n = 256
    shape = (n, n, n)
    sp = [2 * math.pi / n] * 3
    dt0 = 0.8 * sp[0] / 2.0
    dt = 100 * dt0 / 22                                        # Courant numbers up to 3.64
    phi = W.random_modes(shape, W.draw_modes(3, 32, 8, seed=0), device=DEV, dtype=torch.float32)
    vel = W.abc_velocity(shape, device=DEV, dtype=torch.float32)
    out = sl.advect_wide(phi, vel, dt, sp, "CEC", parity)
    torch.cuda.synchronize()
    assert sl.sl_device_status() == 0
    cells = sample_cells(shape, 120, seed=31 + parity)
    r = 15
    wp = windows(phi, cells, r).cpu().double().numpy()
    wv = windows(vel, cells, r).cpu().numpy()                  # float32, (3, n, 31, 31, 31)
    s32 = np.float32(dt / sp[0])
    ref = np.empty(len(cells))
    for i in range(len(cells)):
        c = np.stack([(wv[d, i] * s32).astype(np.float64) for d in range(3)])
        assert np.abs(c).max() < 3.7
        ref[i] = O.step(wp[i], c, O.CEC_SL, parity)[r, r, r]
    got = out[cells[:, 2], cells[:, 1], cells[:, 0]].cpu().double().numpy()
    assert_parity(got, ref, "f32", f"CFL 3.64 parity {parity}, sampled cells")
