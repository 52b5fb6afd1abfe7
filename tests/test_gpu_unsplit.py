"""Unsplit steps (CIR / FEC / BEC, Sec. 2 eqs. intro:FEC, intro:BEC and the 3D
form of eq. CIR2D) on the FP32 3D grids of the four-cell-group CIR kernel's
domain (x a multiple of 4, at least 40; y at least one tile) against the FP64
oracle, cell by cell, on grids with ragged tiles and periodic seams, under a
smooth flow (most warps of the CIR kernel take the packed form on shared
stencil rows) and a random one (most take the per-cell form); and the property
that lets the two forms coexist: a cell's result does not depend on which form
its warp took (for FEC and BEC, on the generic kernel: on velocities beyond the
scheme's reach)."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import assert_parity, oracle_step, random_case
from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
UNSPLIT = ["CIR", "FEC", "BEC"]
# (nz, ny, nx): x a multiple of 4 and >= 48, y >= 16 + 3 (the kernel's domain);
# ragged x and y tiles, tiny and odd z, y shorter than two tiles
SHAPES = [(7, 19, 48), (23, 36, 100), (40, 20, 52), (5, 64, 64), (1, 33, 96), (2, 50, 60)]


def smooth_case(shape, seed, cfl=0.9):
    """ABC velocity scaled to CFL `cfl` and a random-mode field on the shape."""
    nz, ny, nx = shape
    phi = W.random_modes(shape, W.draw_modes(3, 8, 3, seed=seed), dtype=torch.float32)
    vel = W.abc_velocity(shape, dtype=torch.float32)
    sp = [2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz]
    dt = cfl * min(sp) / 2.0
    return phi, vel, sp, dt


@pytest.mark.parametrize("scheme", UNSPLIT)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("flow", ["smooth", "random"])
def test_fast_unsplit_matches_oracle(shape, scheme, flow):
    if flow == "smooth":
        phi, vel, sp, dt = smooth_case(shape, seed=sum(shape))
    else:
        phi, vel, sp, dt = random_case(shape, seed=sum(shape) + 1, dtype="f32")
    out = sl.advect(phi.to(DEV), vel.to(DEV), dt, sp, scheme, 0)
    torch.cuda.synchronize()
    assert sl.sl_device_status() == 0
    ref = oracle_step(phi, vel, sp, dt, scheme, 0)
    assert_parity(out.cpu().numpy(), ref, "f32", f"{scheme} {flow} {shape}")


@pytest.mark.parametrize("scheme", UNSPLIT)
def test_constant_field_is_preserved_bitwise_on_four_cell_groups(scheme):
    shape = (9, 40, 64)
    for phi_v, (_, vel, sp, dt) in ((0.375, smooth_case(shape, 1)), (-2.5, random_case(shape, 5, dtype="f32"))):
        phi = torch.full(shape, phi_v, dtype=torch.float32)
        out = sl.advect(phi.to(DEV), vel.to(DEV), dt, sp, scheme, 0).cpu()
        assert torch.equal(out, phi)


def _dilate(mask, r):
    """Cells within r of a marked cell along every axis (periodic)."""
    out = mask.copy()
    for ax in range(3):
        acc = out.copy()
        for s in range(1, r + 1):
            acc |= np.roll(out, s, axis=ax) | np.roll(out, -s, axis=ax)
        out = acc
    return out


@pytest.mark.parametrize("scheme", UNSPLIT)
def test_result_does_not_depend_on_the_form_a_warp_takes(scheme):
    """A smooth flow, then the same flow with the x velocity negated on a sparse
    set of cells: every warp whose groups contain such a cell switches from the
    packed form to the per-cell form.  Cells whose result cannot depend on the
    changed velocities (beyond the scheme's reach: 0 cells for CIR, 2 for FEC,
    3 for BEC, plus the cells themselves) must come out bitwise equal."""
    shape = (24, 48, 96)
    phi, vel, sp, dt = smooth_case(shape, seed=11)
    rng = np.random.default_rng(3)
    flip = rng.random(shape) < 2e-3
    vel2 = vel.clone()
    vel2[0][torch.from_numpy(flip)] *= -1.0
    a = sl.advect(phi.to(DEV), vel.to(DEV), dt, sp, scheme, 0).cpu().numpy()
    b = sl.advect(phi.to(DEV), vel2.to(DEV), dt, sp, scheme, 0).cpu().numpy()
    reach = {"CIR": 0, "FEC": 2, "BEC": 3}[scheme]
    keep = ~_dilate(flip, reach)
    assert keep.mean() > 0.3
    same = a[keep].view(np.uint32) == b[keep].view(np.uint32)
    assert same.all(), f"{(~same).sum()} of {same.size} cells differ"
    assert not np.array_equal(a, b)
