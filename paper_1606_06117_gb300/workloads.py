"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws and evaluates input fields (initial scalars and
velocities) and the exact solutions of the analytic workloads (the initial
field carried along exact trajectories); it holds none of the advection
schemes' arithmetic.  It serves both the
CUDA path and the FP64 oracle, so that both see the same input values.

All generators evaluate on cell centres x_i = (i + 1/2) * L / N of a periodic
box [0, L)^d and return torch tensors shaped ``(nz, ny, nx)`` (``(ny, nx)`` in
2D, ``(nx,)`` in 1D), x fastest.  Velocities are returned as one tensor with a
leading axis of ``ndim`` components ordered x, y, z (structure of arrays).
Random draws use a seeded numpy generator on the host, so a given seed gives
the same modes on every machine; the fields are then evaluated in float64 on
the requested device and cast to ``dtype``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

TWO_PI = 2.0 * math.pi


def _coords(shape, length, device):
    """1D float64 coordinate vectors (x, y, z order) of the cell centres."""
    dims = list(shape)[::-1]
    return [(torch.arange(n, dtype=torch.float64, device=device) + 0.5) * (length / n) for n in dims]


def _mesh(shape, length, device):
    """Broadcastable coordinate tensors for a (z, y, x) shaped grid, returned as (x, y, z)."""
    c = _coords(shape, length, device)
    nd = len(shape)
    out = []
    for d, v in enumerate(c):
        view = [1] * nd
        view[nd - 1 - d] = -1
        out.append(v.view(view))
    return out


def gaussian(shape, center, sigma, length=1.0, images=1, device="cpu", dtype=torch.float64):
    """exp(-|x - c|^2 / (2 sigma^2)), amplitude 1, summed over periodic images
    within +-``images`` boxes on every axis so the field is periodic."""
    xs = _mesh(shape, length, device)
    out = torch.zeros(shape, dtype=torch.float64, device=device)
    nd = len(shape)
    shifts = np.array(np.meshgrid(*[np.arange(-images, images + 1)] * nd, indexing="ij")).reshape(nd, -1).T
    for sh in shifts:
        r2 = 0.0
        for d in range(nd):
            r2 = r2 + (xs[d] - center[d] - sh[d] * length) ** 2
        out = out + torch.exp(-r2 / (2.0 * sigma * sigma))
    return out.to(dtype)


def gaussian_unwrapped(shape, center, sigma, length=1.0, device="cpu", dtype=torch.float64):
    """exp(-|x - c|^2 / (2 sigma^2)) without periodic images (a blob far from the edges)."""
    return gaussian(shape, center, sigma, length, images=0, device=device, dtype=dtype)


@dataclass
class Modes:
    """A sum of real Fourier modes  sum_m a_m cos(k_m . x + p_m)  on [0, L)^d."""
    k: np.ndarray      # (m, d) integer wavevectors (axis order x, y, z)
    amp: np.ndarray    # (m,)
    phase: np.ndarray  # (m,)


def draw_modes(ndim=3, nmodes=32, kmax=8, seed=0, amp_range=(0.5, 1.0)):
    """nmodes distinct nonzero integer wavevectors with |k| <= kmax, amplitudes
    uniform in amp_range and phases uniform in [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    ks = []
    seen = set()
    while len(ks) < nmodes:
        k = tuple(int(v) for v in rng.integers(-kmax, kmax + 1, size=ndim))
        if all(v == 0 for v in k) or sum(v * v for v in k) > kmax * kmax or k in seen:
            continue
        seen.add(k)
        ks.append(k)
    amp = rng.uniform(amp_range[0], amp_range[1], size=nmodes)
    phase = rng.uniform(0.0, TWO_PI, size=nmodes)
    return Modes(np.asarray(ks, dtype=np.int64), amp, phase)


def random_modes(shape, modes: Modes, length=TWO_PI, device="cpu", dtype=torch.float64):
    """Evaluate a Modes sum on the grid.  Separable: each mode is the real part
    of a product of 1D complex exponentials, contracted over the mode index."""
    nd = len(shape)
    coords = _coords(shape, length, device)
    m = len(modes.amp)
    coef = torch.as_tensor(modes.amp * np.exp(1j * modes.phase), dtype=torch.complex128, device=device)
    fac = []
    for d in range(nd):
        kd = torch.as_tensor(modes.k[:, d], dtype=torch.float64, device=device).view(m, 1)
        fac.append(torch.exp(1j * (TWO_PI / length) * kd * coords[d].view(1, -1)))  # (m, n_d)
    if nd == 1:
        f = torch.einsum("m,mx->x", coef, fac[0])
    elif nd == 2:
        f = torch.einsum("m,my,mx->yx", coef, fac[1], fac[0])
    else:
        f = torch.einsum("m,mz,my,mx->zyx", coef, fac[2], fac[1], fac[0])
    return f.real.contiguous().to(dtype)


def abc_velocity(shape, A=1.0, B=1.0, C=1.0, device="cpu", dtype=torch.float64):
    """Arnold-Beltrami-Childress flow on [0, 2 pi)^3:
    u = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x)."""
    x, y, z = _mesh(shape, TWO_PI, device)
    u = A * torch.sin(z) + C * torch.cos(y) + 0 * x
    v = B * torch.sin(x) + A * torch.cos(z) + 0 * y
    w = C * torch.sin(y) + B * torch.cos(x) + 0 * z
    return torch.stack([u.expand(shape), v.expand(shape), w.expand(shape)]).contiguous().to(dtype)


def taylor_green_velocity(shape, A=1.0, device="cpu", dtype=torch.float64):
    """Taylor-Green vortex on [0, 2 pi)^3: u = A (sin x cos y cos z, -cos x sin y cos z, 0)."""
    x, y, z = _mesh(shape, TWO_PI, device)
    u = A * torch.sin(x) * torch.cos(y) * torch.cos(z)
    v = -A * torch.cos(x) * torch.sin(y) * torch.cos(z)
    w = torch.zeros(shape, dtype=torch.float64, device=device)
    return torch.stack([u.expand(shape), v.expand(shape), w]).contiguous().to(dtype)


def rotation_velocity(shape, device="cpu", dtype=torch.float64):
    """Solid-body rotation about the centre of the unit square: u = 2 pi (0.5 - y, x - 0.5)."""
    x, y = _mesh(shape, 1.0, device)
    u = TWO_PI * (0.5 - y) + 0 * x
    v = TWO_PI * (x - 0.5) + 0 * y
    return torch.stack([u.expand(shape), v.expand(shape)]).contiguous().to(dtype)


def deformation_velocity(shape, device="cpu", dtype=torch.float64):
    """Divergence-free periodic deformation on [0, 1)^3 (to be scaled by cos(pi t / T)):
    u = (2 sin^2(pi x) sin(2 pi y) sin(2 pi z), -sin(2 pi x) sin^2(pi y) sin(2 pi z),
         -sin(2 pi x) sin(2 pi y) sin^2(pi z))."""
    x, y, z = _mesh(shape, 1.0, device)
    sx, sy, sz = torch.sin(math.pi * x), torch.sin(math.pi * y), torch.sin(math.pi * z)
    s2x, s2y, s2z = torch.sin(TWO_PI * x), torch.sin(TWO_PI * y), torch.sin(TWO_PI * z)
    u = 2.0 * sx * sx * s2y * s2z
    v = -s2x * sy * sy * s2z
    w = -s2x * s2y * sz * sz
    return torch.stack([u.expand(shape), v.expand(shape), w.expand(shape)]).contiguous().to(dtype)


# Final time of the patch test (Sec. 5 gives none): the largest speed is
# 3.85e-3, so the patch moves by up to a quarter of the box.
SHEAR_T = 64.0


def shear_profile(s):
    """Velocity profile of the 2D patch test (Sec. 5):
    s (1 - s) (1/2 - s) (cos(2 pi s (1 - s)) + 1) / (2 pi^2)."""
    return s * (1 - s) * (0.5 - s) * (torch.cos(TWO_PI * s * (1 - s)) + 1) / (2 * math.pi ** 2)


def shear_patch_velocity(shape, device="cpu", dtype=torch.float64):
    """The compact divergence-free shear of the paper's 2D patch test (Sec. 5) on
    the unit square: u = profile(y), v = -profile(x)."""
    x, y = _mesh(shape, 1.0, device)
    u = shear_profile(y) + 0 * x
    v = -shear_profile(x) + 0 * y
    return torch.stack([u.expand(shape), v.expand(shape)]).contiguous().to(dtype)


def shear_stream(x, y):
    """Stream function of the patch-test velocity, psi = P(x) + P(y) with
    u = d psi / dy and v = -d psi / dx.  P' = profile integrates in
    w = s (1 - s): P = (w sin(2 pi w) / (2 pi) + cos(2 pi w) / (4 pi^2) + w^2 / 2) / (4 pi^2)."""
    def P(s):
        w = s * (1 - s)
        return (w * torch.sin(TWO_PI * w) / TWO_PI + torch.cos(TWO_PI * w) / (4 * math.pi ** 2) + w * w / 2) / (
            4 * math.pi ** 2)
    return P(x) + P(y)


def shear_departure(x, y, T=SHEAR_T, nsub=512):
    """Exact departure points: where the points (x, y) at time T were at time 0
    under the patch-test velocity, by classical fourth-order Runge-Kutta
    integration backwards in time with nsub steps (FP64), in the periodic box:
    the profile is evaluated at coordinates reduced to [0, 1), and the points
    are returned reduced.  The trajectories are level curves of shear_stream
    (of the periodic box: curves below the saddle value circle the corners)."""
    h = -T / nsub
    x = x.to(torch.float64)
    y = y.to(torch.float64)

    def f(px, py):
        return shear_profile(torch.remainder(py, 1.0)), -shear_profile(torch.remainder(px, 1.0))
    for _ in range(nsub):
        a1, b1 = f(x, y)
        a2, b2 = f(x + 0.5 * h * a1, y + 0.5 * h * b1)
        a3, b3 = f(x + 0.5 * h * a2, y + 0.5 * h * b2)
        a4, b4 = f(x + h * a3, y + h * b3)
        x = x + h / 6 * (a1 + 2 * a2 + 2 * a3 + a4)
        y = y + h / 6 * (b1 + 2 * b2 + 2 * b3 + b4)
    return torch.remainder(x, 1.0), torch.remainder(y, 1.0)


def shear_exact(shape, initial, T=SHEAR_T, nsub=512, device="cpu", dtype=torch.float64):
    """Exact solution of the patch test at time T on the cell centres: the
    initial field initial(x0, y0) (a function of FP64 coordinate tensors) at the
    exact departure points."""
    x, y = _mesh(shape, 1.0, device)
    x, y = torch.broadcast_tensors(x, y)
    x0, y0 = shear_departure(x, y, T, nsub)
    return initial(x0, y0).to(dtype)


def patch_indicator(lo=0.25, hi=0.5):
    """The square patch of Sec. 5 as a function of coordinates: 1 inside [lo, hi)^2."""
    def f(x, y):
        return ((x >= lo) & (x < hi) & (y >= lo) & (y < hi)).to(torch.float64)
    return f


def bump(center=(0.375, 0.375), sigma=0.06):
    """A smooth Gaussian in the patch's place, exp(-|x - c|^2 / (2 sigma^2)), for
    convergence orders under the same flow (below 4e-9 at the box edges)."""
    def f(x, y):
        return torch.exp(-((x - center[0]) ** 2 + (y - center[1]) ** 2) / (2 * sigma * sigma))
    return f


def square_patch(shape, lo=0.25, hi=0.5, device="cpu", dtype=torch.float64):
    """1 inside the square [lo, hi)^2, 0 outside (Sec. 5 patch test)."""
    x, y = _mesh(shape, 1.0, device)
    return patch_indicator(lo, hi)(*torch.broadcast_tensors(x, y)).to(dtype)


def on_grid(shape, f, device="cpu", dtype=torch.float64):
    """A function of FP64 coordinate tensors (x, y) evaluated on the 2D cell centres."""
    x, y = _mesh(shape, 1.0, device)
    return f(*torch.broadcast_tensors(x, y)).to(dtype)


def profile_1d(n, kind, device="cpu", dtype=torch.float64):
    """The 1D initial profiles of Sec. 4 on [0, 1): 'heaviside' sgn(sin 2 pi x),
    'triangle' |x - 0.5|, 'cosine' -cos(2 pi x)."""
    (x,) = _coords((n,), 1.0, device)
    if kind == "heaviside":
        f = torch.sign(torch.sin(TWO_PI * x))
    elif kind == "triangle":
        f = (x - 0.5).abs()
    elif kind == "cosine":
        f = -torch.cos(TWO_PI * x)
    else:
        raise ValueError(kind)
    return f.to(dtype)


def dt_for_cfl(total_time, max_speed_over_dx, cfl):
    """Time step that reaches total_time exactly with max |u_d| dt / dx_d <= cfl:
    dt = T / ceil(T * max(|u_d|/dx_d) / cfl).  Returns (dt, nsteps)."""
    nsteps = int(math.ceil(total_time * max_speed_over_dx / cfl - 1e-12))
    return total_time / nsteps, nsteps


@dataclass
class Instance:
    """One member of a batch of independent periodic problems."""
    n: int
    flow: str          # "abc" or "tg"
    amps: tuple        # (A, B, C) for abc, (A,) for tg
    modes_seed: int


def draw_batch(count=48, sizes=(64, 96, 128, 160, 192), seed=0):
    """count instances with cubic sizes drawn uniformly from ``sizes``, each with
    a Taylor-Green or ABC velocity whose amplitudes are uniform in [0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        if rng.random() < 0.5:
            out.append(Instance(n, "abc", tuple(float(a) for a in rng.uniform(0.5, 1.5, 3)), seed * 1000 + i))
        else:
            out.append(Instance(n, "tg", (float(rng.uniform(0.5, 1.5)),), seed * 1000 + i))
    return out


def instance_fields(inst: Instance, device="cpu", dtype=torch.float32, nmodes=32, kmax=8):
    """(scalar, velocity) of one batch instance on [0, 2 pi)^3."""
    shape = (inst.n,) * 3
    phi = random_modes(shape, draw_modes(3, nmodes, kmax, inst.modes_seed), device=device, dtype=dtype)
    if inst.flow == "abc":
        vel = abc_velocity(shape, *inst.amps, device=device, dtype=dtype)
    else:
        vel = taylor_green_velocity(shape, inst.amps[0], device=device, dtype=dtype)
    return phi, vel


# ------------------------------------------------------------- Rayleigh-Benard
def rb_spots(nx, nz, Lx=2.0, Lz=1.0, amp=0.1, r=0.1, hot=(0.25, 0.2), cold=(0.5, 0.2)):
    """The start of the Sec. 6 runs: a hot spot (theta = +amp) next to a cold
    spot (theta = -amp) near the lower left corner of the box [0, Lx] x [0, Lz]
    (walls, not periodic), U = 0.  Here disks of radius r (in units of Lz)
    centred at ``hot`` and ``cold``, on the cell centres of nx x nz cells;
    returns a (nz, nx) float64 numpy array."""
    x = (np.arange(nx) + 0.5) * (Lx / nx)
    z = (np.arange(nz) + 0.5) * (Lz / nz)
    X, Z = np.meshgrid(x, z)
    th = np.zeros((nz, nx))
    th[(X - hot[0]) ** 2 + (Z - hot[1]) ** 2 < r ** 2] = amp
    th[(X - cold[0]) ** 2 + (Z - cold[1]) ** 2 < r ** 2] = -amp
    return th
