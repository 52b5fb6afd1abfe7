"""The Rayleigh-Benard box on the GPU (sl_rb_*, Sec. 6) against the FP64
oracle of the same discretisation, cell by cell, for every scheme, on grids
with several kernel tiles and ragged edges; and the properties the equations
fix: the rest state stays exactly at rest, a conduction eigenmode decays by
the discrete heat factor, a mirror-symmetric start stays mirror-symmetric.

Tolerance: the two sides solve the Poisson equation differently (a dense
eigen-decomposition pseudo-inverse in the oracle, the cosine eigenbasis here),
so their projections differ by a few eps * kappa of the zero-mean Neumann
Laplacian (kappa = lam_max / lam_min); the cell-by-cell bound per step is
max(1e-12, 8 eps kappa) of max |oracle| in FP64, and max(1e-5, 8 eps32 kappa)
in FP32."""
import numpy as np
import pytest
import torch

from gpu_helpers import assert_parity
from oracle import rb_oracle as R
from paper_1606_06117_gb300 import workloads as W
from paper_1606_06117_gb300 import _lib as sl

pytestmark = pytest.mark.gpu
SCHEMES = ["CIR", "FEC", "BEC", "CEC"]


def kappa(nx, nz, Lx=2.0, Lz=1.0):
    dx, dz = Lx / nx, Lz / nz
    lmax = 4 / dx ** 2 + 4 / dz ** 2
    lmin = min(4 / dx ** 2 * np.sin(np.pi / (2 * nx)) ** 2, 4 / dz ** 2 * np.sin(np.pi / (2 * nz)) ** 2)
    return lmax / lmin


def allowance(nx, nz, steps, f64=True):
    eps, base = (np.finfo(np.float64).eps, 1e-12) if f64 else (np.finfo(np.float32).eps, 1e-5)
    return steps * max(1.0, 8 * eps * kappa(nx, nz) / base)


def plume_start(nx, nz, seed):
    rng = np.random.default_rng(seed)
    th = W.rb_spots(nx, nz) + 0.01 * rng.standard_normal((nz, nx))
    return np.zeros((nz, nx)), np.zeros((nz, nx)), th


def random_start(nx, nz, seed, cmax, dt, Lx=2.0, Lz=1.0):
    """Velocities with per-cell random signs up to Courant cmax (every upwind branch)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-cmax, cmax, (nz, nx)) * (Lx / nx) / dt
    w = rng.uniform(-cmax, cmax, (nz, nx)) * (Lz / nz) / dt
    return u, w, 0.1 * rng.standard_normal((nz, nx))


def run_both(nx, nz, scheme, start, dt, steps, Ra, dtype=torch.float64, Pr=1.0):
    box = R.Box(nx, nz, Ra=Ra, Pr=Pr, scheme=scheme)
    box.u, box.w, box.theta = (np.array(a, dtype=np.float64) for a in start)
    if dtype == torch.float32:   # the oracle starts from the values the GPU receives
        box.u, box.w, box.theta = (a.astype(np.float32).astype(np.float64) for a in (box.u, box.w, box.theta))
    g = sl.RayleighBenard(nx, nz, Ra=Ra, Pr=Pr, scheme=scheme, dtype=dtype)
    try:
        sl.sl_device_status()
        g.set_state(*(torch.from_numpy(np.ascontiguousarray(a)) for a in start))
        for _ in range(steps):
            box.step(dt)
        g.step(dt, steps)
        got = [t.cpu().double().numpy() for t in g.state()]
        torch.cuda.synchronize()
        assert sl.sl_device_status() == 0
    finally:
        g.close()
    return got, [box.u, box.w, box.theta]


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("nx,nz,steps", [(16, 8, 12), (24, 12, 7), (37, 19, 4), (50, 50, 3)])
def test_plume_steps_match_the_oracle(scheme, nx, nz, steps):
    got, ref = run_both(nx, nz, scheme, plume_start(nx, nz, seed=nx), 2e-4, steps, Ra=1e5)
    for name, a, b in zip(("u", "w", "theta"), got, ref):
        assert_parity(a, b, "f64", f"{scheme} {nx}x{nz} {name}", allowance(nx, nz, steps))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_the_papers_run_matches_the_oracle_after_a_thousand_steps(scheme):
    """The Sec. 6 run at its size: 50 x 50 cells, Ra = 1e5, Pr = 1, the +-0.1
    spots, 1000 steps of dt = 2e-5 (the plume reaches the top).  This flow does
    not amplify rounding differences over the run (in the oracle, a relative
    1e-13 perturbation of theta is still 1e-13 after 1000 steps), so the bound
    is ten single-step bounds, not a thousand."""
    got, ref = run_both(50, 50, scheme, (np.zeros((50, 50)), np.zeros((50, 50)), W.rb_spots(50, 50)), 2e-5, 1000,
                        Ra=1e5)
    for name, a, b in zip(("u", "w", "theta"), got, ref):
        assert_parity(a, b, "f64", f"{scheme} 50x50 x1000 {name}", allowance(50, 50, 10))
    assert (got[2][-3:] > 0.02).any()


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("nx,nz", [(16, 8), (29, 13)])
def test_random_high_courant_steps_match_the_oracle(scheme, nx, nz):
    """Two steps from velocities of random sign per cell, Courant up to 0.45
    (both CEC sweep orders; the forces keep the second step's Courant below 1)."""
    dt = 1e-5
    got, ref = run_both(nx, nz, scheme, random_start(nx, nz, seed=nz, cmax=0.45, dt=dt), dt, 2, Ra=1e4)
    for name, a, b in zip(("u", "w", "theta"), got, ref):
        assert_parity(a, b, "f64", f"{scheme} {nx}x{nz} {name}", allowance(nx, nz, 2))


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("Pr", [0.7, 4.0])
def test_prandtl_numbers_other_than_one_match_the_oracle(scheme, Pr):
    """Pr multiplies both the buoyancy and the viscous term (eq. e:nsnd); a
    random start exercises both from the first step."""
    nx, nz, dt = 24, 12, 2e-5
    u, w, th = random_start(nx, nz, seed=7, cmax=0.2, dt=dt)
    got, ref = run_both(nx, nz, scheme, (u, w, th), dt, 4, Ra=3e4, Pr=Pr)
    for name, a, b in zip(("u", "w", "theta"), got, ref):
        assert_parity(a, b, "f64", f"{scheme} Pr {Pr} {name}", allowance(nx, nz, 4))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_float32_box_tracks_the_oracle(scheme):
    nx, nz, steps = 32, 16, 5
    got, ref = run_both(nx, nz, scheme, plume_start(nx, nz, seed=3), 2e-4, steps, Ra=1e5, dtype=torch.float32)
    for name, a, b in zip(("u", "w", "theta"), got, ref):
        assert_parity(a, b, "f32", f"{scheme} f32 {name}", allowance(nx, nz, steps, f64=False))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_rest_state_stays_exactly_at_rest(scheme):
    g = sl.RayleighBenard(20, 10, Ra=1e6, scheme=scheme)
    try:
        g.step(1e-4, 5)
        assert all(not t.any() for t in g.state())
    finally:
        g.close()


@pytest.mark.parametrize("j,k", [(0, 1), (2, 1), (1, 3)])
def test_conduction_mode_decays_by_the_discrete_heat_factor(j, k):
    nx, nz, dt = 16, 8, 1e-4
    dx, dz = 2.0 / nx, 1.0 / nz
    v = np.outer(np.sin(np.pi * k * (np.arange(nz) + 0.5) / nz), np.cos(np.pi * j * (np.arange(nx) + 0.5) / nx))
    lam = -4 / dx ** 2 * np.sin(np.pi * j / (2 * nx)) ** 2 - 4 / dz ** 2 * np.sin(np.pi * k / (2 * nz)) ** 2
    g = sl.RayleighBenard(nx, nz, Ra=0.0, scheme="CEC")
    try:
        z = torch.zeros((nz, nx), dtype=torch.float64)
        g.set_state(z, z, torch.from_numpy(v))
        g.step(dt, 10)
        u, w, th = (t.cpu().numpy() for t in g.state())
    finally:
        g.close()
    assert np.allclose(th, (1 + dt * lam) ** 10 * v, rtol=0, atol=1e-12)
    assert not u.any() and not w.any()


@pytest.mark.parametrize("scheme", ["CIR", "CEC"])
def test_mirror_symmetric_start_stays_mirror_symmetric(scheme):
    nx, nz = 20, 10
    th = W.rb_spots(nx, nz, hot=(1.0, 0.25), cold=(1.0, 0.6), r=0.15)
    th = 0.5 * (th + th[:, ::-1])
    g = sl.RayleighBenard(nx, nz, Ra=5e4, scheme=scheme)
    try:
        z = torch.zeros((nz, nx), dtype=torch.float64)
        g.set_state(z, z, torch.from_numpy(np.ascontiguousarray(th)))
        g.step(2e-4, 8)
        u, w, th = (t.cpu().numpy() for t in g.state())
    finally:
        g.close()
    assert np.abs(w).max() > 1e-3
    for f, s in ((th, 1), (w, 1), (u, -1)):
        assert np.allclose(f, s * f[:, ::-1], rtol=0, atol=1e-12 * max(1.0, np.abs(f).max()))


@pytest.mark.parametrize("scheme", ["FEC", "CEC"])
def test_graph_replayed_runs_equal_single_steps_bitwise(scheme):
    """Runs of 16 steps or more replay captured CUDA graphs of 8 steps; they
    give the single-step launches' results bit for bit, from an odd step, for
    a run that ends on a partial graph, and after dt changes (a new capture)."""
    nx, nz = 24, 12
    _, _, th = plume_start(nx, nz, seed=5)
    z = torch.zeros((nz, nx), dtype=torch.float64)
    a = sl.RayleighBenard(nx, nz, Ra=1e5, scheme=scheme)
    b = sl.RayleighBenard(nx, nz, Ra=1e5, scheme=scheme)
    try:
        for g in (a, b):
            g.set_state(z, z, torch.from_numpy(th))
        plan = [(2e-4, 1), (2e-4, 37), (1.5e-4, 20), (1.5e-4, 16), (2e-4, 3)]
        for dt, k in plan:
            a.step(dt, k)
            for _ in range(k):
                b.step(dt, 1)
        for x, y in zip(a.state(), b.state()):
            assert torch.equal(x, y)
    finally:
        a.close()
        b.close()


def test_state_round_trip_and_argument_errors():
    g = sl.RayleighBenard(12, 6)
    try:
        a = [torch.randn((6, 12), dtype=torch.float64) for _ in range(3)]
        g.set_state(*a)
        assert all(torch.equal(x.cuda(), y) for x, y in zip(a, g.state()))
        with pytest.raises(sl.SLError):
            sl.sl_rb_step(g.h, float("nan"))
        with pytest.raises(sl.SLError):
            sl.sl_rb_step(g.h, 1e-4, -1)
    finally:
        g.close()
    for bad in ((3, 8), (8, 3), (5000, 8)):
        with pytest.raises(sl.SLError):
            sl.sl_rb_create(*bad)
    with pytest.raises(sl.SLError):
        sl.sl_rb_create(8, 8, Lx=0.0)
    with pytest.raises(sl.SLError):
        sl.sl_rb_create(8, 8, dtype=sl.F32_D64)


@pytest.mark.parametrize("nx,nz,dt", [(4, 4, 1e-3), (4096, 48, 2e-8)])
def test_smallest_and_largest_boxes_keep_the_mirror_symmetry(nx, nz, dt):
    """The box's extreme sizes (4 cells per axis; 4096 cells along x, where the
    transforms sum 4096 terms) against a property that holds at any size: a
    start symmetric about x = Lx / 2 stays symmetric (theta, w even, u odd).
    The bound allows the transforms' rounding, 1e-11 of the field's maximum."""
    x = (np.arange(nx) + 0.5) * (2.0 / nx)
    zc = (np.arange(nz) + 0.5) / nz
    th = 0.1 * np.outer(np.sin(np.pi * zc), np.cos(np.pi * x) + 0.5 * np.cos(3 * np.pi * x))
    th = 0.5 * (th + th[:, ::-1])
    g = sl.RayleighBenard(nx, nz, Ra=1e5, scheme="CEC")
    try:
        z = torch.zeros((nz, nx), dtype=torch.float64)
        g.set_state(z, z, torch.from_numpy(np.ascontiguousarray(th)))
        sl.sl_device_status()
        g.step(dt, 3)
        u, w, th = (t.cpu().numpy() for t in g.state())
        assert sl.sl_device_status() == 0
    finally:
        g.close()
    assert np.isfinite(u).all() and np.isfinite(w).all() and np.isfinite(th).all()
    assert np.abs(w).max() > 0
    for f, s in ((th, 1), (w, 1), (u, -1)):
        assert np.allclose(f, s * f[:, ::-1], rtol=0, atol=1e-11 * np.abs(f).max())


def test_boxes_of_different_sizes_step_side_by_side():
    """Two live boxes whose transforms stage different amounts of shared memory
    (80 x 40: 79.5 KB, 24 x 12: 9 KB), created large first, stepped in turn:
    each gives the result it gives alone."""
    def start(nx, nz):
        u, w, th = plume_start(nx, nz, seed=nx)
        return [torch.from_numpy(np.ascontiguousarray(a)) for a in (u, w, th)]
    solo = {}
    for nx, nz in ((80, 40), (24, 12)):
        g = sl.RayleighBenard(nx, nz, Ra=1e5, scheme="CEC")
        try:
            g.set_state(*start(nx, nz))
            g.step(2e-5, 20)
            solo[nx] = g.state()
        finally:
            g.close()
    a = sl.RayleighBenard(80, 40, Ra=1e5, scheme="CEC")
    b = sl.RayleighBenard(24, 12, Ra=1e5, scheme="CEC")
    try:
        a.set_state(*start(80, 40))
        b.set_state(*start(24, 12))
        for _ in range(4):
            b.step(2e-5, 5)
            a.step(2e-5, 5)
        for x, y in zip(a.state(), solo[80]):
            assert torch.equal(x, y)
        for x, y in zip(b.state(), solo[24]):
            assert torch.equal(x, y)
    finally:
        a.close()
        b.close()


def test_steps_on_a_side_stream_equal_steps_on_the_default_stream():
    """sl_rb_step enqueues on the caller's stream (eager kernels and replayed
    graphs alike); a box stepped on a side stream ends where the same box
    stepped on the default stream does."""
    nx, nz = 24, 12
    u, w, th = plume_start(nx, nz, seed=9)
    start = [torch.from_numpy(np.ascontiguousarray(a)) for a in (u, w, th)]
    res = []
    for use_side in (False, True):
        g = sl.RayleighBenard(nx, nz, Ra=1e5, scheme="CEC")
        try:
            g.set_state(*start)
            if use_side:
                s = torch.cuda.Stream()
                with torch.cuda.stream(s):
                    g.step(2e-5, 3)
                    g.step(2e-5, 24)
                    out = g.state()
                s.synchronize()
            else:
                g.step(2e-5, 3)
                g.step(2e-5, 24)
                out = g.state()
                torch.cuda.synchronize()
            res.append([t.clone() for t in out])
        finally:
            g.close()
    for x, y in zip(*res):
        assert torch.equal(x, y)
