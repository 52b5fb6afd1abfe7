"""FP64 CPU oracle of the Rayleigh-Benard driver of Sec. 6 (eqs. e:nsnd, e:Tnd,
e:mnd, e:poisson, e:proj): semi-Lagrangian advection of the velocity and the
temperature perturbation, explicit buoyancy and diffusion, and a
pressure-correction projection, in a 2D box with walls on all four sides.

TEST INFRASTRUCTURE ONLY (like ``oracle.py``): the tests, ``smoke()`` and the
benchmark's CPU leg may use it; the product path never does.  It shares no code
with the CUDA path.  Plain numpy; the Poisson equation is solved with a dense
pseudo-inverse of the assembled discrete operator (from its symmetric
eigen-decomposition).

Readings (the paper gives the equations, not the discretisation details):
* Grid: nx x nz cells of a box Lx x Lz (the paper's aspect ratio Lz/Lx = 0.5),
  cell-centred, fields as (nz, nx) arrays (x fastest, z upwards).
* Ghost points: G = 3 layers around the box (the reach of the split CEC
  stencil).  No-slip walls: u and w are mirrored with a sign change across
  every wall.  Temperature: theta = 0 on the plates (mirrored with a sign
  change across z = 0 and z = Lz), d theta / dx = 0 on the side walls
  (mirrored without one).  Ghost columns are filled first (interior rows),
  then ghost rows over the full padded width.
* Advection L[f, U^n]: one step of the chosen scheme of the paper (CIR, FEC,
  BEC, or the split CEC with sweep order alternating with the step index) on
  the padded grid with the padded velocity U^n, whose wrap-around only ever
  reaches ghost cells; only the interior is kept.
* Forces: second-order finite-volume Laplacians of the step-n fields (5-point
  stencil with the ghost values), all explicit:
    u2 = L[u] + dt Pr lap u,  w2 = L[w] + dt (Ra Pr theta + Pr lap w),
    theta_new = L[theta] + dt (w + lap theta)
  (eq. e:nsnd has Pr lap U; the printed discrete step drops the factor Pr,
  which is taken as a misprint).
* Projection: face velocities are the averages of the two adjacent cells, zero
  on the walls (impermeability); their finite-volume divergence D is the
  right-hand side of lap phi = D with the compact 5-point Laplacian and
  d phi / dn = 0 on the walls (ghost phi mirrored), zero mean.  The faces are
  corrected by the face gradient of phi (then exactly divergence-free) and
  the cell velocities by the average of their two faces' corrections.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

G = 3


def pad(f):
    nz, nx = f.shape
    p = np.zeros((nz + 2 * G, nx + 2 * G))
    p[G:G + nz, G:G + nx] = f
    return p


def fill(p, sx, sz):
    """Ghost layers of a padded field in place: mirror across the side walls
    with sign sx, across the plates with sign sz."""
    nz, nx = p.shape[0] - 2 * G, p.shape[1] - 2 * G
    for j in range(G):
        p[G:G + nz, G - 1 - j] = sx * p[G:G + nz, G + j]
        p[G:G + nz, G + nx + j] = sx * p[G:G + nz, G + nx - 1 - j]
    for j in range(G):
        p[G - 1 - j, :] = sz * p[G + j, :]
        p[G + nz + j, :] = sz * p[G + nz - 1 - j, :]
    return p


def laplacian(p, dx, dz):
    """5-point Laplacian at the interior cells of a padded field."""
    nz, nx = p.shape[0] - 2 * G, p.shape[1] - 2 * G
    c = p[G:G + nz, G:G + nx]
    return ((p[G:G + nz, G + 1:G + nx + 1] - 2 * c + p[G:G + nz, G - 1:G + nx - 1]) / dx ** 2 +
            (p[G + 1:G + nz + 1, G:G + nx] - 2 * c + p[G - 1:G + nz - 1, G:G + nx]) / dz ** 2)


def poisson_matrix(nx, nz, dx, dz):
    """The discrete Neumann Laplacian as a dense (nz nx) x (nz nx) matrix."""
    n = nx * nz
    A = np.zeros((n, n))
    for k in range(nz):
        for i in range(nx):
            r = k * nx + i
            for di, dk, h in ((1, 0, dx), (-1, 0, dx), (0, 1, dz), (0, -1, dz)):
                ii, kk = i + di, k + dk
                if 0 <= ii < nx and 0 <= kk < nz:   # a wall neighbour is the mirror: no flux
                    A[r, kk * nx + ii] += 1 / h ** 2
                    A[r, r] -= 1 / h ** 2
    return A


def neumann_pinv(A):
    """Pseudo-inverse of the symmetric discrete Neumann Laplacian from its
    eigen-decomposition: the one zero eigenvalue (constant eigenvector) is
    dropped, so solutions have zero mean."""
    lam, V = np.linalg.eigh(A)
    keep = np.abs(lam) > 1e-9 * np.abs(lam).max()
    assert keep.sum() == len(lam) - 1, "the Neumann Laplacian has exactly one zero eigenvalue"
    return (V[:, keep] / lam[keep]) @ V[:, keep].T


class Box:
    """One Rayleigh-Benard run: state (u, w, theta) as (nz, nx) float64 arrays."""

    def __init__(self, nx, nz, Lx=2.0, Lz=1.0, Ra=1e5, Pr=1.0, scheme="CEC"):
        self.nx, self.nz, self.dx, self.dz = nx, nz, Lx / nx, Lz / nz
        self.Ra, self.Pr, self.scheme = Ra, Pr, O.SCHEMES[scheme]
        self.pinv = neumann_pinv(poisson_matrix(nx, nz, self.dx, self.dz))
        self.u = np.zeros((nz, nx))
        self.w = np.zeros((nz, nx))
        self.theta = np.zeros((nz, nx))
        self.n = 0

    def solve(self, rhs):
        """Zero-mean solution of lap phi = rhs with d phi / dn = 0."""
        return (self.pinv @ rhs.ravel()).reshape(rhs.shape)

    def divergence(self, u2, w2):
        """Face velocities (cell averages, zero on the walls) and their divergence."""
        uf = np.zeros((self.nz, self.nx + 1))
        wf = np.zeros((self.nz + 1, self.nx))
        uf[:, 1:-1] = 0.5 * (u2[:, :-1] + u2[:, 1:])
        wf[1:-1, :] = 0.5 * (w2[:-1, :] + w2[1:, :])
        return uf, wf, (uf[:, 1:] - uf[:, :-1]) / self.dx + (wf[1:, :] - wf[:-1, :]) / self.dz

    def step(self, dt):
        dx, dz, Ra, Pr = self.dx, self.dz, self.Ra, self.Pr
        pu = fill(pad(self.u), -1, -1)
        pw = fill(pad(self.w), -1, -1)
        pt = fill(pad(self.theta), 1, -1)
        C = np.stack([pu * (dt / dx), pw * (dt / dz)])
        adv = [O.step(f, C, self.scheme, self.n)[G:G + self.nz, G:G + self.nx] for f in (pu, pw, pt)]
        u2 = adv[0] + dt * Pr * laplacian(pu, dx, dz)
        w2 = adv[1] + dt * (Ra * Pr * self.theta + Pr * laplacian(pw, dx, dz))
        theta = adv[2] + dt * (self.w + laplacian(pt, dx, dz))
        uf, wf, div = self.divergence(u2, w2)
        phi = self.solve(div)
        gx = np.zeros((self.nz, self.nx + 1))
        gz = np.zeros((self.nz + 1, self.nx))
        gx[:, 1:-1] = (phi[:, 1:] - phi[:, :-1]) / dx
        gz[1:-1, :] = (phi[1:, :] - phi[:-1, :]) / dz
        self.u = u2 - 0.5 * (gx[:, :-1] + gx[:, 1:])
        self.w = w2 - 0.5 * (gz[:-1, :] + gz[1:, :])
        self.theta = theta
        self.n += 1
        # the projected faces, for the divergence pin
        return uf - gx, wf - gz

