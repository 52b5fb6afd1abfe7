"""The Sec. 5 patch test through the CUDA path: a 2D field under the paper's
compact divergence-free shear, compared with the initial field carried along
exact trajectories (workloads.shear_exact).  Multi-step parity with the oracle
at 128^2, and at 256^2 / 512^2 (where the oracle would take minutes) the
paper's ranking on the discontinuous patch and the constant-velocity orders
1 / 2 / 2 / 3 on a smooth field under the same flow (Sec. 5)."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import assert_parity
from oracle import oracle as O
from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
SCHEMES = ["CIR", "FEC", "BEC", "CEC"]


def gpu_run(n, initial, scheme, dtype):
    """The patch test at n^2, CFL 0.5, to W.SHEAR_T; returns (final field, the
    velocity the kernels saw, dt, steps)."""
    shape = (n, n)
    sl.sl_device_status()   # clears the status word
    t = torch.float64 if dtype == "f64" else torch.float32
    vel = W.shear_patch_velocity(shape, device=DEV).to(t)
    dt, nsteps = W.dt_for_cfl(W.SHEAR_T, vel.abs().max().item() * n, 0.5)
    x = W.on_grid(shape, initial, device=DEV).to(t)
    y = torch.empty_like(x)
    code, dc = getattr(sl, scheme), (sl.F64 if dtype == "f64" else sl.F32)
    for k in range(nsteps):
        sl.sl_advect(y, x, vel, 2, [n, n, 1], [1.0 / n, 1.0 / n, 1.0], dt, code, dc, k & 1)
        x, y = y, x
    torch.cuda.synchronize()
    assert sl.sl_device_status() == 0
    return x, vel, dt, nsteps


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_patch_test_matches_the_oracle(scheme, dtype):
    n = 128
    got, vel, dt, nsteps = gpu_run(n, W.patch_indicator(), scheme, dtype)
    c = vel.double().cpu().numpy() * (dt * n)
    ref = O.run(W.on_grid((n, n), W.patch_indicator()).numpy(), c, O.SCHEMES[scheme], nsteps)
    assert_parity(got.cpu().numpy(), ref, dtype, f"patch test {scheme} {dtype}",
                  allowance=(nsteps if dtype == "f64" else 4))


def test_patch_ranking_at_512():
    """Figs. dis1 / dis2: CIR farthest from the exact solution, CEC closest."""
    n = 512
    exact = W.shear_exact((n, n), W.patch_indicator(), device=DEV)
    l1 = {s: (gpu_run(n, W.patch_indicator(), s, "f64")[0] - exact).abs().mean().item() for s in SCHEMES}
    assert l1["CEC"] < l1["BEC"] < l1["FEC"] < l1["CIR"], l1


def test_smooth_field_orders_256_to_512():
    lo = {"CIR": 0.8, "FEC": 1.85, "BEC": 1.85, "CEC": 2.6}
    hi = {"CIR": 1.2, "FEC": 2.2, "BEC": 2.2, "CEC": 3.3}
    errs = {}
    for n in (256, 512):
        exact = W.shear_exact((n, n), W.bump(), device=DEV)
        for s in SCHEMES:
            got = gpu_run(n, W.bump(), s, "f64")[0]
            errs[(s, n)] = (torch.linalg.vector_norm(got - exact) / torch.linalg.vector_norm(exact)).item()
    for s in SCHEMES:
        order = math.log2(errs[(s, 256)] / errs[(s, 512)])
        assert lo[s] < order < hi[s], (s, order, errs)
    assert errs[("CEC", 512)] < errs[("BEC", 512)] < errs[("FEC", 512)] < errs[("CIR", 512)]
