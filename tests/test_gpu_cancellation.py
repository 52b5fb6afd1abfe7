"""Cancellation stress for the round-trip difference delta = Phi - Phi_bar
(Sec. 2): a field of 1000 plus perturbations of 1e-3, with Courant numbers
clustered near 0, 1/2 and 1 where delta is smallest against Phi.  Each result
is compared cell by cell with the FP64 oracle on the same (float-rounded)
inputs, for float storage and arithmetic (delta from neighbour differences),
float storage with delta in double, and double throughout.  The float paths
must stay within a few units in the last place of the field's magnitude: delta
enters the result additively, so forming it in float does not cost accuracy
beyond the rounding of the stored field."""
import numpy as np
import pytest
import torch

from gpu_helpers import courant, oracle_step
from paper_1606_06117_gb300 import _lib as sl

pytestmark = pytest.mark.gpu
DEV = "cuda"
ULP_1000 = 2.0 ** -14          # spacing of float32 numbers in [512, 1024)


def stress_case(shape, seed, centre, dtype):
    rng = np.random.default_rng(seed)
    phi = 1000.0 + 1e-3 * rng.standard_normal(shape)
    sign = rng.choice([-1.0, 1.0], size=(3,) + shape)
    C = sign * np.clip(centre + 1e-3 * rng.standard_normal((3,) + shape), 0.0, 1.0)
    sp, dt = [1.0, 1.0, 1.0], 1.0
    t = torch.float64 if dtype == "f64" else torch.float32
    return torch.from_numpy(phi).to(t), torch.from_numpy(C).to(t), sp, dt


@pytest.mark.parametrize("centre", [1e-3, 0.5, 1.0 - 1e-3])
@pytest.mark.parametrize("scheme", ["FEC", "BEC", "CEC"])
@pytest.mark.parametrize("dtype", ["f32", "f32_d64", "f64"])
@pytest.mark.parametrize("shape", [(12, 20, 28), (16, 32, 64)])
def test_cancellation_stress(shape, dtype, scheme, centre):
    phi, vel, sp, dt = stress_case(shape, 11, centre, dtype)
    for parity in ((0, 1) if scheme == "CEC" else (0,)):
        out = sl.advect(phi.to(DEV), vel.to(DEV), dt, sp, scheme, parity, delta64=(dtype == "f32_d64"))
        ref = oracle_step(phi, vel, sp, dt, scheme, parity)
        err = np.abs(out.cpu().double().numpy() - ref).max()
        bound = 1e-12 if dtype == "f64" else 4 * ULP_1000
        print(f"{scheme} {dtype} C~{centre} {shape} parity {parity}: max |GPU - oracle| = {err:.3e} "
              f"({err / ULP_1000:.2f} ulp of 1000)")
        assert err <= bound, (err, bound)
