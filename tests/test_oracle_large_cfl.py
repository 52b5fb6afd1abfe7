"""Large Courant numbers (Sec. 3 on BEC stability, Sec. 4 eq. intro:CECcoefSL):
pins of the oracle's non-local schemes and of the paper's stability statement.

- Non-local interpolation (the corners bracket the departure point, however
  far) makes integer Courant numbers exact shifts for every scheme.
- The adopted large-CFL CEC (correction at the departure cell) is, for constant
  velocity, the upwind cubic Lagrange interpolation at the departure point (a
  textbook routine written out here), and stays third order.
- The literal reading (only the weights change) has the closed-form symbol
  built from the operator definitions, and falls to second order: the reason
  it is not the adopted one.
- Local stencils beyond U = 1 (the paper's BEC remark): the printed xi_B is
  bounded by 1 up to U = 1.5 and not beyond; CIR, FEC and CEC are unstable as
  soon as U > 1.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1606_06117_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_1d_constant_u.json")))
LARGE = [O.CIR, O.FEC, O.BEC, O.CEC_SL, O.CEC_SL_LIT]


def ev(expr, **kw):
    env = {"cos": np.cos, "sin": np.sin, "exp": np.exp}
    env.update(kw)
    return eval(expr, env)  # noqa: S307 - committed fixture


def cubic_lagrange_at(phi, X):
    """Periodic 4-point Lagrange interpolation of phi at positions X (cell units),
    through the nodes floor(X) - 1 .. floor(X) + 2."""
    n = len(phi)
    b = np.floor(X).astype(np.int64)
    t = X - b                                   # in [0, 1)
    nodes = [-1.0, 0.0, 1.0, 2.0]
    out = np.zeros_like(X, dtype=np.float64)
    for k, xk in enumerate(nodes):
        w = np.ones_like(t)
        for xj in nodes:
            if xj != xk:
                w *= (t - xj) / (xk - xj)
        out += w * phi[(b - 1 + k) % n]
    return out


@pytest.mark.parametrize("scheme", LARGE)
def test_integer_courant_is_an_exact_shift(scheme):
    shape = (6, 7, 9)
    rng = np.random.default_rng(21)
    phi = rng.standard_normal(shape)
    c = np.stack([np.full(shape, v) for v in (3.0, -2.0, 1.0)])
    out = O.step(phi, c, scheme, 0)
    assert np.array_equal(out, np.roll(phi, shift=(1, -2, 3), axis=(0, 1, 2)))


@pytest.mark.parametrize("C", [0.4, -0.7, 1.3, 2.75, 3.75, -2.3, -3.6, 5.2])
def test_large_cfl_cec_is_cubic_lagrange_at_the_departure_point(C):
    n = 37
    rng = np.random.default_rng(22)
    phi = rng.standard_normal(n)
    got = O.step(phi, np.full((1, n), C), O.CEC_SL, 0)
    want = cubic_lagrange_at(phi, np.arange(n) - C)
    assert np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("parity", [0, 1])
def test_large_cfl_cec_3d_is_tricubic(parity):
    """Constant velocity, split sweeps: the tensor product of the 1D cubic
    interpolations at the departure point, in either sweep order."""
    shape = (7, 8, 9)
    rng = np.random.default_rng(23)
    phi = rng.standard_normal(shape)
    C = (2.6, -1.35, 3.2)                      # x, y, z
    got = O.step(phi, np.stack([np.full(shape, v) for v in C]), O.CEC_SL, parity)
    want = phi
    for axis, cv in enumerate(C):               # axis 0 = x = array axis 2
        arr = np.moveaxis(want, 2 - axis, -1)
        n = arr.shape[-1]
        arr = np.apply_along_axis(lambda line: cubic_lagrange_at(line, np.arange(n) - cv), -1, arr)
        want = np.moveaxis(arr, -1, 2 - axis)
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("C", [1.3, 2.75, 3.75, -2.3])
@pytest.mark.parametrize("k", [1, 4, 9])
def test_literal_large_cfl_cec_symbol(C, k):
    """a FEC + b BEC with the operator definitions and 3a = 2 - 1/(U % 1): for
    constant velocity L_U = shift(m) * local L at the fraction f, the round
    trip cancels the shift, delta has the symbol d = 1 - |l|^2, FEC = e l + d/2,
    BEC = e l (1 + d/2)."""
    n = 48
    th = 2 * math.pi * k / n
    U, sgn = abs(C), (1 if C > 0 else -1)
    m, f = math.floor(U), U - math.floor(U)
    e = np.exp(-1j * sgn * m * th)
    lam = 1 - f + f * np.exp(-1j * sgn * th)
    d = 1 - abs(lam) ** 2
    a = (2 - 1 / f) / 3
    want = a * (e * lam + d / 2) + (1 - a) * e * lam * (1 + d / 2)
    j = np.arange(n)
    c = np.full((1, n), C)
    got = O.step(np.cos(j * th), c, O.CEC_SL_LIT) + 1j * O.step(np.sin(j * th), c, O.CEC_SL_LIT)
    assert np.max(np.abs(got / np.exp(1j * j * th) - want)) < 1e-13


def translation_errors(scheme, cfl, sizes=(128, 256, 512)):
    errs = []
    for n in sizes:
        phi0 = W.gaussian((n,), [0.5], 0.1, images=2).numpy()
        dt, nsteps = W.dt_for_cfl(1.0, n, cfl)
        c = np.full((1, n), dt * n)
        phi = O.run(phi0, c, scheme, nsteps)
        exact = phi0                          # once around the periodic interval
        errs.append(O.norms(phi, exact)[0])
    return errs


@pytest.mark.parametrize("scheme,lo,hi", [(O.CIR, 0.8, 1.2), (O.FEC, 1.8, 2.3), (O.BEC, 1.8, 2.3),
                                          (O.CEC_SL, 2.8, 3.3), (O.CEC_SL_LIT, 1.8, 2.3)])
@pytest.mark.parametrize("cfl", [2.3, 3.75])
def test_large_cfl_orders(scheme, cfl, lo, hi):
    """Translation once around the unit interval at CFL 2.3 and 3.75: CIR 1,
    FEC / BEC 2, the adopted CEC 3 (accuracy preserved, as Sec. 4 states); the
    literal reading only 2."""
    e = translation_errors(scheme, cfl)
    order = math.log2(e[-2] / e[-1])
    assert lo < order < hi, (scheme, cfl, e)


def test_sampled_cells_reject_large_courant():
    phi = np.zeros((8, 8))
    c = np.full((2, 8, 8), 1.5)
    with pytest.raises(RuntimeError):
        O.sample(phi, c, O.CIR, 0, [[1, 2, 0]])


def test_local_stencils_beyond_cfl_one():
    """Sec. 3: with the local stencil (the neighbours i and i - s, extrapolating
    beyond U = 1), BEC stays stable up to U = 1.5 and the other schemes do not
    survive U > 1.  The printed xi_B is bounded by 1 exactly up to 1.5."""
    af = GOLD["amplification_factors"]
    th = np.linspace(1e-4, math.pi, 4001)

    def peak(name, U):
        if name == "CIR":
            return np.abs(1 - U + U * np.exp(-1j * th)).max()
        return np.abs(ev(af[name]["expr"], U=U, th=th)).max()
    for U in (1.05, 1.2, 1.4, 1.5):
        assert peak("BEC", U) <= 1 + 1e-12, U
    for U in (1.51, 1.6):
        assert peak("BEC", U) > 1.05, U
    for name in ("CIR", "FEC", "CEC_reading"):
        assert peak(name, 1.05) > 1.05, name


@pytest.mark.parametrize("shape", [(29,), (9, 14), (5, 6, 7)])
def test_large_cfl_cec_equals_the_local_cec_below_cfl_one(shape):
    """With m = trunc(C) = 0 the departure cell is the arrival cell: the adopted
    large-CFL CEC is the local CEC (R7) operation for operation, bit for bit."""
    rng = np.random.default_rng(24)
    phi = rng.standard_normal(shape)
    c = rng.uniform(-0.99, 0.99, size=(len(shape),) + shape)
    for parity in (0, 1):
        assert np.array_equal(O.step(phi, c, O.CEC_SL, parity), O.step(phi, c, O.CEC, parity))
