"""Convergence orders and the paper's qualitative rankings, on the FP64 oracle.

The schemes converge with orders 1 / 2 / 2 / 3 (CIR / FEC / BEC / CEC, Sec. 3
and Table 1) on a smooth Gaussian under refinement; translations at a constant non-aligned
velocity have exact trajectories, so the error is the scheme's own.
"""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1606_06117_gb300 import workloads as W


def translate_error(scheme, n, ndim, vel, cfl, sigma, T=1.0):
    shape = (n,) * ndim
    center = [0.5] * ndim
    phi0 = W.gaussian(shape, center, sigma, images=2).numpy()
    dt, nsteps = W.dt_for_cfl(T, max(abs(v) for v in vel) * n, cfl)
    c = np.stack([np.full(shape, v * dt * n) for v in vel])
    phi = O.run(phi0, c, scheme, nsteps)
    shifted = [(ctr + v * T) % 1.0 for ctr, v in zip(center, vel)]
    exact = W.gaussian(shape, shifted, sigma, images=2).numpy()
    return O.norms(phi, exact)[0]


def orders(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("scheme,lo,hi", [(O.CIR, 0.85, 1.15), (O.FEC, 1.85, 2.2),
                                          (O.BEC, 1.85, 2.2), (O.CEC, 2.8, 3.2)])
def test_orders_1d_translation(scheme, lo, hi):
    errs = [translate_error(scheme, n, 1, (1.0,), 0.37, 0.15 if scheme == O.CIR else 0.08)
            for n in (128, 256, 512)]
    assert all(lo < p < hi for p in orders(errs)), orders(errs)


@pytest.mark.parametrize("scheme,lo,hi", [(O.FEC, 1.8, 2.25), (O.BEC, 1.8, 2.25), (O.CEC, 2.7, 3.25)])
def test_orders_2d_translation(scheme, lo, hi):
    errs = [translate_error(scheme, n, 2, (1.0, 0.6), 0.8, 0.1) for n in (32, 64, 128)]
    p = orders(errs)
    assert lo < p[-1] < hi, p


def test_cir_first_order_2d():
    errs = [translate_error(O.CIR, n, 2, (1.0, 0.6), 0.8, 0.2) for n in (64, 128, 256)]
    p = orders(errs)
    assert 0.8 < p[-1] < 1.15, p


def rotation_errors(n, schemes):
    """Config-1 style: Gaussian (sigma 0.05 at (0.25, 0.5)) under solid-body rotation,
    CFL 0.5, one revolution; error against the initial (= exact) field."""
    shape = (n, n)
    phi0 = W.gaussian_unwrapped(shape, (0.25, 0.5), 0.05).numpy()
    vel = W.rotation_velocity(shape).numpy()
    dt, nsteps = W.dt_for_cfl(1.0, math.pi * n, 0.5)
    c = vel * dt * n
    out = {}
    for s in schemes:
        out[s] = O.norms(O.run(phi0, c, s, nsteps), phi0)
    return out


def test_rotation_ranking():
    """Sec. 5 / Sec. 6: CEC closest to the exact solution, CIR farthest."""
    e = rotation_errors(64, [O.CIR, O.FEC, O.BEC, O.CEC])
    l2 = {s: v[0] for s, v in e.items()}
    assert l2[O.CEC] < l2[O.BEC] < l2[O.FEC] < l2[O.CIR]


@pytest.mark.parametrize("kind", ["heaviside", "triangle"])
def test_1d_profiles_cec_closest(kind):
    """Sec. 4 (figs. 1Dhea, 1Dtri): N = 30, CFL 0.75, 10 periods; CEC is the scheme
    closest to the analytic solution."""
    n = 30
    phi0 = W.profile_1d(n, kind).numpy()
    nsteps = int(round(10 * n / 0.75))
    c = np.full((1, n), 0.75)
    err = {s: O.norms(O.run(phi0, c, s, nsteps), phi0)[0] for s in (O.CIR, O.FEC, O.BEC, O.CEC)}
    assert err[O.CEC] == min(err.values())


def test_time_reversal_flow_returns():
    """Config-5 style: the deformation flow scaled by cos(pi t / T) brings every
    field back at t = T; the CEC error falls with resolution."""
    errs = []
    for n in (16, 32):
        shape = (n, n, n)
        phi0 = W.random_modes(shape, W.draw_modes(3, 4, 2, seed=3), length=1.0).numpy()
        vel = W.deformation_velocity(shape).numpy()
        nsteps = 2 * n
        T = 1.0
        dt = T / nsteps
        phi = phi0
        for k in range(nsteps):
            scale = math.cos(math.pi * (k + 0.5) * dt / T)
            phi = O.step(phi, vel * (dt * scale * n), O.CEC, parity=k)
        errs.append(O.norms(phi, phi0)[2])
    assert errs[1] < errs[0] / 2.5, errs


def test_workload_dt_hits_final_time():
    dt, n = W.dt_for_cfl(1.0, math.pi * 128, 0.5)
    assert n == 805 and n * dt == pytest.approx(1.0)


def test_random_modes_are_seeded_and_periodic():
    m = W.draw_modes(3, 32, 8, seed=0)
    assert len({tuple(k) for k in m.k}) == 32 and np.all((m.k ** 2).sum(1) <= 64)
    a = W.random_modes((8, 8, 8), m).numpy()
    b = W.random_modes((8, 8, 8), W.draw_modes(3, 32, 8, seed=0)).numpy()
    assert np.array_equal(a, b)
    # direct evaluation of one cell
    x = (np.array([2, 5, 7]) + 0.5) * 2 * math.pi / 8
    ref = sum(am * math.cos(float(k @ x) + p) for k, am, p in zip(m.k, m.amp, m.phase))
    assert a[7, 5, 2] == pytest.approx(ref, abs=1e-12)
    assert torch.is_tensor(W.abc_velocity((4, 4, 4)))


# ------------------------------------------------------- Sec. 5 patch test (E5)
def shear_case(n):
    """Grid Courant numbers and step count of the patch test at n^2, CFL 0.5,
    final time W.SHEAR_T (reached exactly)."""
    shape = (n, n)
    vel = W.shear_patch_velocity(shape).numpy()
    dt, nsteps = W.dt_for_cfl(W.SHEAR_T, np.abs(vel).max() * n, 0.5)
    return vel * (dt * n), nsteps


def shear_errors(n, initial):
    """(L1, relative L2) of each scheme's oracle solution against the initial
    field carried along exact trajectories."""
    shape = (n, n)
    c, nsteps = shear_case(n)
    phi0 = W.on_grid(shape, initial).numpy()
    exact = W.shear_exact(shape, initial).numpy()
    out = {}
    for s in (O.CIR, O.FEC, O.BEC, O.CEC):
        phi = O.run(phi0, c, s, nsteps)
        out[s] = (np.abs(phi - exact).mean(), O.norms(phi, exact)[2])
    return out


def test_shear_reference_trajectories():
    """The exact-trajectory reference of the patch test: the departure points
    keep the closed-form stream function psi = P(x) + P(y) of the flow, whose
    derivatives are the velocity of Sec. 5 (u = d psi / dy, v = -d psi / dx);
    integrating forward again returns to the start; halving the Runge-Kutta
    step changes nothing at 1e-9."""
    x, y = torch.meshgrid(torch.linspace(0.01, 0.99, 41, dtype=torch.float64),
                          torch.linspace(0.02, 0.98, 37, dtype=torch.float64), indexing="xy")
    h = 1e-6
    dpsi_dy = (W.shear_stream(x, y + h) - W.shear_stream(x, y - h)) / (2 * h)
    dpsi_dx = (W.shear_stream(x + h, y) - W.shear_stream(x - h, y)) / (2 * h)
    assert torch.allclose(dpsi_dy, W.shear_profile(y), atol=1e-9, rtol=0)
    assert torch.allclose(-dpsi_dx, -W.shear_profile(x), atol=1e-9, rtol=0)
    x0, y0 = W.shear_departure(x, y)
    assert (W.shear_stream(x0, y0) - W.shear_stream(x, y)).abs().max() < 1e-11
    x1, y1 = W.shear_departure(x0, y0, T=-W.SHEAR_T)

    def pdist(a, b):
        d = (a - b).abs()
        return torch.minimum(d, 1 - d).max()
    assert pdist(x1, x) < 1e-9 and pdist(y1, y) < 1e-9
    x2, y2 = W.shear_departure(x, y, nsub=1024)
    assert pdist(x2, x0) < 1e-9 and pdist(y2, y0) < 1e-9
    assert pdist(x0, x) > 0.1            # the flow does move the points


def test_shear_patch_ranking():
    """Sec. 5 (figs. dis1, dis2): on the discontinuous square patch CIR has the
    largest error and CEC the smallest; the four schemes rank
    CEC < BEC < FEC < CIR at two resolutions."""
    for n in (64, 128):
        e = {s: v[0] for s, v in shear_errors(n, W.patch_indicator()).items()}
        assert e[O.CEC] < e[O.BEC] < e[O.FEC] < e[O.CIR], (n, e)


def test_shear_smooth_field_orders():
    """Sec. 5: for regularly varying velocities the orders are those of constant
    velocity, 1 / 2 / 2 / 3: a Gaussian in the patch's place, same flow, exact
    trajectories, 64^2 -> 128^2."""
    lo = {O.CIR: 0.7, O.FEC: 1.8, O.BEC: 1.8, O.CEC: 2.6}
    hi = {O.CIR: 1.3, O.FEC: 2.3, O.BEC: 2.3, O.CEC: 3.4}
    e64, e128 = shear_errors(64, W.bump()), shear_errors(128, W.bump())
    for s in lo:
        order = math.log2(e64[s][1] / e128[s][1])
        assert lo[s] < order < hi[s], (s, order)
