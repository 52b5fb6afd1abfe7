"""Pins of the Rayleigh-Benard oracle (Sec. 6) against what the mathematics
fixes: the discrete operators' closed-form eigenpairs, exact divergence-free
projected faces, the conductive rest state, exact decay of a conduction
eigenmode, and the box's left-right mirror symmetry."""
import numpy as np
import pytest

from oracle import rb_oracle as R
from paper_1606_06117_gb300 import workloads as W


def test_ghost_fill_mirrors_across_each_wall():
    f = np.arange(1.0, 1 + 6 * 8).reshape(6, 8)
    p = R.fill(R.pad(f), sx=1, sz=-1)
    G = R.G
    for j in range(G):
        assert np.array_equal(p[G:G + 6, G - 1 - j], p[G:G + 6, G + j])            # even across x = 0
        assert np.array_equal(p[G:G + 6, G + 8 + j], p[G:G + 6, G + 7 - j])        # even across x = Lx
        assert np.array_equal(p[G - 1 - j, :], -p[G + j, :])                       # odd across z = 0
        assert np.array_equal(p[G + 6 + j, :], -p[G + 5 - j, :])                   # odd across z = Lz


@pytest.mark.parametrize("j,k", [(0, 1), (3, 0), (2, 5), (7, 3)])
def test_neumann_laplacian_has_the_cosine_eigenpairs(j, k):
    """The cell-centred Neumann Laplacian is diagonalised by
    cos(pi j (i + 1/2) / nx) cos(pi k (m + 1/2) / nz), with eigenvalue
    -(4 / dx^2) sin^2(pi j / 2 nx) - (4 / dz^2) sin^2(pi k / 2 nz)."""
    nx, nz, dx, dz = 12, 8, 2.0 / 12, 1.0 / 8
    A = R.poisson_matrix(nx, nz, dx, dz)
    v = np.outer(np.cos(np.pi * k * (np.arange(nz) + 0.5) / nz), np.cos(np.pi * j * (np.arange(nx) + 0.5) / nx))
    lam = -4 / dx ** 2 * np.sin(np.pi * j / (2 * nx)) ** 2 - 4 / dz ** 2 * np.sin(np.pi * k / (2 * nz)) ** 2
    assert np.allclose(A @ v.ravel(), lam * v.ravel(), atol=1e-10)
    box2 = R.Box.__new__(R.Box)
    box2.pinv = R.neumann_pinv(A)
    phi = box2.solve(lam * v)
    assert np.allclose(phi, v, atol=1e-10)


def test_projected_faces_are_divergence_free_and_mean_zero_phi():
    rng = np.random.default_rng(1)
    box = R.Box(16, 8, Ra=2e4, scheme="CEC")
    box.theta = 0.1 * rng.standard_normal((8, 16))
    box.u = 0.5 * rng.standard_normal((8, 16))
    box.w = 0.5 * rng.standard_normal((8, 16))
    for _ in range(3):
        uf, wf = box.step(2e-4)
        div = (uf[:, 1:] - uf[:, :-1]) / box.dx + (wf[1:, :] - wf[:-1, :]) / box.dz
        scale = np.abs(uf).max() / box.dx
        assert np.abs(div).max() <= 1e-11 * scale
        assert np.all(uf[:, 0] == 0) and np.all(uf[:, -1] == 0) and np.all(wf[0] == 0) and np.all(wf[-1] == 0)


@pytest.mark.parametrize("scheme", ["CIR", "FEC", "BEC", "CEC"])
def test_conductive_rest_state_stays_exactly_at_rest(scheme):
    box = R.Box(16, 8, Ra=1e6, scheme=scheme)
    for _ in range(5):
        box.step(1e-4)
    assert not box.u.any() and not box.w.any() and not box.theta.any()


@pytest.mark.parametrize("j,k", [(0, 1), (2, 1), (1, 3)])
def test_conduction_mode_decays_by_the_discrete_heat_factor(j, k):
    """U = 0 and Ra = 0: theta obeys theta_new = (1 + dt lam) theta for a
    discrete conduction eigenmode cos(pi j (i + 1/2) / nx) sin(pi k (m + 1/2) / nz)
    (d theta / dx = 0 on the side walls, theta = 0 on the plates)."""
    nx, nz, dt = 16, 8, 1e-4
    box = R.Box(nx, nz, Ra=0.0, scheme="CEC")
    v = np.outer(np.sin(np.pi * k * (np.arange(nz) + 0.5) / nz), np.cos(np.pi * j * (np.arange(nx) + 0.5) / nx))
    lam = -4 / box.dx ** 2 * np.sin(np.pi * j / (2 * nx)) ** 2 - 4 / box.dz ** 2 * np.sin(np.pi * k / (2 * nz)) ** 2
    box.theta = v.copy()
    for _ in range(10):
        box.step(dt)
    assert np.allclose(box.theta, (1 + dt * lam) ** 10 * v, rtol=0, atol=1e-12)
    assert not box.u.any() and not box.w.any()


@pytest.mark.parametrize("scheme", ["CIR", "CEC"])
def test_mirror_symmetric_start_stays_mirror_symmetric(scheme):
    """theta symmetric about x = Lx / 2 and U = 0: theta and w stay symmetric
    and u antisymmetric (the box and the equations are invariant under x -> Lx - x)."""
    nx, nz = 20, 10
    th = W.rb_spots(nx, nz, hot=(1.0, 0.25), cold=(1.0, 0.6), r=0.15)
    th = 0.5 * (th + th[:, ::-1])                     # exactly symmetric (x_i - 1 rounds unevenly)
    assert np.array_equal(th, th[:, ::-1]) and th.any()
    box = R.Box(nx, nz, Ra=5e4, scheme=scheme)
    box.theta = th
    for _ in range(8):
        box.step(2e-4)
    assert np.abs(box.w).max() > 1e-3
    for f, s in ((box.theta, 1), (box.w, 1), (box.u, -1)):
        assert np.allclose(f, s * f[:, ::-1], rtol=0, atol=1e-12 * max(1.0, np.abs(f).max()))


def test_buoyancy_lifts_the_hot_spot():
    """A hot spot starts rising: after a few steps w > 0 over it, w < 0 over the cold one."""
    nx, nz = 24, 12
    box = R.Box(nx, nz, Ra=1e5, scheme="CEC")
    box.theta = W.rb_spots(nx, nz)
    for _ in range(10):
        box.step(1e-4)
    x = (np.arange(nx) + 0.5) * box.dx
    z = (np.arange(nz) + 0.5) * box.dz
    ih, ic, kz = np.argmin(np.abs(x - 0.25)), np.argmin(np.abs(x - 0.5)), np.argmin(np.abs(z - 0.2))
    assert box.w[kz, ih] > 0 > box.w[kz, ic]


def test_one_step_from_rest_scales_with_ra_pr():
    """From U = 0 the first step has no advection and no viscous term, so the
    new velocity is the projection of dt Ra Pr theta e_z: linear in Ra Pr
    (eq. e:nsnd's buoyancy carries both factors), and theta does not depend on
    them."""
    nx, nz = 16, 8
    th = W.rb_spots(nx, nz, hot=(0.5, 0.4), cold=(1.2, 0.5), r=0.2)
    runs = {}
    for Ra, Pr in ((1e4, 1.0), (1e4, 2.5), (2.5e4, 1.0)):
        box = R.Box(nx, nz, Ra=Ra, Pr=Pr, scheme="CEC")
        box.theta = th.copy()
        box.step(1e-4)
        runs[(Ra, Pr)] = (box.u, box.w, box.theta)
    u1, w1, t1 = runs[(1e4, 1.0)]
    assert np.abs(w1).max() > 0
    for key in ((1e4, 2.5), (2.5e4, 1.0)):
        u, w, t = runs[key]
        assert np.allclose(u, 2.5 * u1, rtol=0, atol=1e-12 * np.abs(u).max())
        assert np.allclose(w, 2.5 * w1, rtol=0, atol=1e-12 * np.abs(w).max())
        assert np.array_equal(t, t1)


def test_viscous_term_is_linear_in_pr():
    """With Ra = 0 and theta = 0 one step from a velocity field differs from
    the Pr = 0 step by Pr times the (projected) viscous increment dt lap U;
    theta, which gains dt w from the base-state gradient (eq. e:Tnd), does not
    depend on Pr."""
    rng = np.random.default_rng(3)
    nx, nz = 16, 8
    u0, w0 = 0.3 * rng.standard_normal((nz, nx)), 0.3 * rng.standard_normal((nz, nx))
    out = {}
    for Pr in (0.0, 1.0, 0.7):
        box = R.Box(nx, nz, Ra=0.0, Pr=Pr, scheme="FEC")
        box.u, box.w = u0.copy(), w0.copy()
        box.step(1e-4)
        out[Pr] = (box.u, box.w, box.theta)
    assert np.array_equal(out[0.7][2], out[0.0][2]) and np.abs(out[0.0][2]).max() > 0
    for k in range(2):
        inc = out[1.0][k] - out[0.0][k]
        assert np.abs(inc).max() > 1e-6
        assert np.allclose(out[0.7][k] - out[0.0][k], 0.7 * inc, rtol=0, atol=1e-12)
