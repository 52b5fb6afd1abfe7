"""Solid-body rotation of a Gaussian (Sec. 5 and Sec. 6 comparisons; the 2D
FP64 workload: sigma 0.05 at (0.25, 0.5), u = 2 pi (0.5 - y, x - 0.5), CFL 0.5,
one revolution) advanced by the CUDA path for all four schemes: every result
matches the FP64 oracle's, and the error against the exact (initial) field
ranks CEC < BEC < FEC < CIR."""
import math

import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2
from oracle import oracle as O
from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
SCHEMES = (("CIR", O.CIR), ("FEC", O.FEC), ("BEC", O.BEC), ("CEC", O.CEC))


@pytest.mark.parametrize("n", [64, 128])
def test_rotation_matches_oracle_and_ranks(n):
    shape = (n, n)
    phi0 = W.gaussian_unwrapped(shape, (0.25, 0.5), 0.05)
    vel = W.rotation_velocity(shape)
    dt, nsteps = W.dt_for_cfl(1.0, math.pi * n, 0.5)
    sp = [1.0 / n, 1.0 / n]
    c = vel.numpy() * dt * n
    err = {}
    for name, code in SCHEMES:
        x, v = phi0.to(DEV), vel.to(DEV)
        y = torch.empty_like(x)
        for k in range(nsteps):
            sl.advect(x, v, dt, sp, name, k, out=y)
            x, y = y, x
        gpu = x.cpu().numpy()
        ref = O.run(phi0.numpy(), c, code, nsteps)
        # FP64, 1e-12 per step from identical inputs; the schemes do not amplify
        # (|g| <= 1), so rounding differences add up at most linearly over the run
        assert rel_l2(gpu, ref) <= 1e-12 * nsteps, name
        err[name] = rel_l2(gpu, phi0.numpy())
    assert err["CEC"] < err["BEC"] < err["FEC"] < err["CIR"], err
