"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed stencils, amplification factors and modified-equation coefficients
(tests/golden/paper_1d_constant_u.json, transcribed from Sec. 3 and Table 1),
textbook routines (cubic Lagrange interpolation), exact shifts, constants and a
brute-force matrix composition built from the paper's explicit CIR formula
(eq. CIR2D) rather than from the oracle's floor/fraction form.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_1d_constant_u.json")))
ALL = [O.CIR, O.FEC, O.BEC, O.CEC]
NAMES = {O.CIR: "CIR", O.FEC: "FEC", O.BEC: "BEC", O.CEC: "CEC"}


def ev(expr, **kw):
    env = {"cos": np.cos, "sin": np.sin, "exp": np.exp}
    env.update(kw)
    return eval(expr, env)  # noqa: S307 - committed fixture


def const_courant(shape, values):
    return np.stack([np.full(shape, v, dtype=np.float64) for v in values])


def symbol(scheme, U, theta, n=64, probe=5):
    """One-step amplification of exp(i j theta) by the oracle (u > 0 when U > 0)."""
    j = np.arange(n)
    c = np.full((1, n), U)
    a = O.step(np.cos(j * theta), c, scheme)
    b = O.step(np.sin(j * theta), c, scheme)
    return ((a + 1j * b) / np.exp(1j * j * theta))[probe]


# --------------------------------------------------------------------------- P1
@pytest.mark.parametrize("scheme", ALL)
@pytest.mark.parametrize("shape", [(33,), (9, 14), (5, 6, 7)])
def test_constant_field_is_preserved(scheme, shape):
    """Any velocity and scheme keep a constant field constant (weights sum to 1)."""
    rng = np.random.default_rng(1)
    c = rng.uniform(-1, 1, size=(len(shape),) + shape)
    out = O.step(np.full(shape, 2.75), c, scheme, parity=1)
    assert np.max(np.abs(out - 2.75)) <= 8 * np.finfo(float).eps * 2.75


# --------------------------------------------------------------------------- P2
@pytest.mark.parametrize("scheme", ALL)
@pytest.mark.parametrize("cvals", [(1.0, -1.0, 0.0), (1.0, 1.0, 1.0), (-1.0, 0.0, 1.0)])
def test_integer_courant_is_an_exact_shift(scheme, cvals):
    """At integer Courant numbers every scheme is the exact cyclic shift, bitwise."""
    shape = (6, 7, 8)
    phi = np.random.default_rng(2).standard_normal(shape)
    out = O.step(phi, const_courant(shape, cvals), scheme, parity=0)
    ref = np.roll(phi, shift=(int(cvals[2]), int(cvals[1]), int(cvals[0])), axis=(0, 1, 2))
    assert np.array_equal(out, ref)


# --------------------------------------------------------------------------- P3
@pytest.mark.parametrize("U", [0.13, 0.37, 0.5, 0.81, 1.0])
@pytest.mark.parametrize("name", ["FEC", "BEC"])
def test_1d_constant_velocity_stencils_match_paper(name, U):
    """FEC = eq. cstUHALO, BEC = eq. cstUBEC (Sec. 3) for a constant velocity."""
    n = 40
    phi = np.random.default_rng(3).standard_normal(n)
    out = O.step(phi, np.full((1, n), U), O.SCHEMES[name])
    ref = sum(ev(e, U=U) * np.roll(phi, -int(o)) for o, e in GOLD["stencils"][name]["coeffs"].items())
    # the departure point i - U is rounded at the scale of i, hence n * eps
    assert np.max(np.abs(out - ref)) < 1e-13


def test_fec_constant_velocity_is_lax_wendroff():
    """For constant velocity FEC with CIR is the Lax-Wendroff stencil (textbook)."""
    n, U = 50, 0.42
    phi = np.random.default_rng(4).standard_normal(n)
    lw = phi - U / 2 * (np.roll(phi, -1) - np.roll(phi, 1)) + U * U / 2 * (np.roll(phi, -1) - 2 * phi + np.roll(phi, 1))
    assert np.max(np.abs(O.step(phi, np.full((1, n), U), O.FEC) - lw)) < 1e-14


def lagrange_weights(t, nodes):
    return [np.prod([(t - m) / (k - m) for m in nodes if m != k]) for k in nodes]


@pytest.mark.parametrize("C", [0.11, 0.37, 0.5, 0.93, -0.29, -0.77])
def test_1d_cec_is_upwind_cubic_lagrange(C):
    """Constant velocity CEC = cubic Lagrange interpolation at i - C on the four
    upwind-biased nodes (i-2..i+1 for C > 0, i-1..i+2 for C < 0)."""
    n = 37
    phi = np.random.default_rng(5).standard_normal(n)
    out = O.step(phi, np.full((1, n), C), O.CEC)
    nodes = [-2, -1, 0, 1] if C > 0 else [-1, 0, 1, 2]
    ref = sum(w * np.roll(phi, -k) for w, k in zip(lagrange_weights(-C, nodes), nodes))
    assert np.max(np.abs(out - ref)) < 1e-13


@pytest.mark.parametrize("parity", [0, 1])
def test_3d_split_cec_constant_velocity_is_tricubic(parity):
    """With a constant velocity the split CEC step is the tensor-product tricubic
    Lagrange interpolation, whatever the sweep order."""
    shape = (7, 8, 9)
    cv = (0.31, -0.62, 0.77)
    phi = np.random.default_rng(6).standard_normal(shape)
    out = O.step(phi, const_courant(shape, cv), O.CEC, parity=parity)
    ref = np.zeros(shape)
    axes_nodes = [[-2, -1, 0, 1] if c > 0 else [-1, 0, 1, 2] for c in cv]
    wts = [lagrange_weights(-c, nd) for c, nd in zip(cv, axes_nodes)]
    for wx, kx in zip(wts[0], axes_nodes[0]):
        for wy, ky in zip(wts[1], axes_nodes[1]):
            for wz, kz in zip(wts[2], axes_nodes[2]):
                ref += wx * wy * wz * np.roll(phi, shift=(-kz, -ky, -kx), axis=(0, 1, 2))
    assert np.max(np.abs(out - ref)) < 1e-13


# --------------------------------------------------------------------------- P4
@pytest.mark.parametrize("U", [0.2, 0.37, 0.8, 0.95])
@pytest.mark.parametrize("k", [1, 3, 7, 13])
def test_amplification_factors_match_paper(U, k):
    """xi_F and xi_B as printed (Sec. 3); xi_C in the reading recorded in the fixture."""
    th = 2 * math.pi * k / 64
    af = GOLD["amplification_factors"]
    assert abs(symbol(O.FEC, U, th) - ev(af["FEC"]["expr"], U=U, th=th)) < 1e-14
    assert abs(symbol(O.BEC, U, th) - ev(af["BEC"]["expr"], U=U, th=th)) < 1e-14
    assert abs(symbol(O.CEC, U, th) - ev(af["CEC_reading"]["expr"], U=U, th=th)) < 1e-14


def test_printed_xi_c_is_not_consistent():
    """The printed xi_C does not tend to exp(-i U th) (wrong first-order phase), which is
    why the fixture records a reading; the reading does."""
    U, th = 0.3, 1e-3
    af = GOLD["amplification_factors"]
    printed = ev(af["CEC_as_printed"]["expr"], U=U, th=th)
    reading = ev(af["CEC_reading"]["expr"], U=U, th=th)
    assert abs(np.angle(printed) + U * th) > 0.5 * th
    assert abs(np.angle(reading) + U * th) < 1e-9


@pytest.mark.parametrize("scheme", ALL)
def test_fourier_mode_closed_form_after_many_steps(scheme):
    """For constant velocity the oracle's n-step result on a single mode is
    Re(g^n exp(i k x)), with g its own one-step symbol (linearity, P4)."""
    n, U, k, steps = 48, 0.61, 5, 400
    th = 2 * math.pi * k / n
    g = symbol(scheme, U, th, n=n)
    j = np.arange(n)
    phi = np.cos(j * th)
    c = np.full((1, n), U)
    for s in range(steps):
        phi = O.step(phi, c, scheme, s)
    assert np.max(np.abs(phi - (g ** steps * np.exp(1j * j * th)).real)) < 1e-11


# --------------------------------------------------------------------------- P6
@pytest.mark.parametrize("U", [0.2, 0.37, 0.8])
def test_modified_equation_coefficients_match_table1(U):
    """The leading modified-equation terms (Sec. 3 / Table 1, App. B decomposition
    of the symbol into decay and phase) match the oracle's exact symbol as k dx -> 0."""
    me = GOLD["modified_equation"]
    u, dx = 1.0, 1.0 / 512
    dt = U * dx / u
    th = 2 * math.pi * 2 / 512
    k = th / dx

    def rate(coeffs):
        return dt * sum(ev(e, U=U, u=u, dx=dx, dt=dt) * (1j * k) ** int(a) for a, e in coeffs.items())

    for name, scheme in (("CIR", O.CIR), ("FEC", O.FEC), ("BEC", O.BEC), ("CEC", O.CEC)):
        lg = np.log(symbol(scheme, U, th, n=512))
        pred = rate(me[name])
        assert lg.real / pred.real == pytest.approx(1.0, abs=2e-3), name
        if name in ("FEC", "BEC"):
            assert (lg.imag + U * th) / pred.imag == pytest.approx(1.0, abs=2e-3), name
        if name == "CEC":   # no third-derivative (dispersive) term
            assert abs(lg.imag + U * th) < 1e-2 * abs(pred.real)


@pytest.mark.parametrize("scheme,alpha", [(O.CIR, 2), (O.FEC, 4), (O.BEC, 4), (O.CEC, 4)])
def test_decay_rate_scales_with_resolution(scheme, alpha):
    """App. B: at fixed CFL, C_alpha ~ N^(1-alpha), so the decay rate sigma of the
    first harmonic times N^(alpha-1) is constant (eq. coefres)."""
    U = 0.37
    vals = []
    for n in (64, 128, 256, 512):
        th = 2 * math.pi / n
        dt = U / n
        sigma = -math.log(abs(symbol(scheme, U, th, n=n))) / dt
        vals.append(sigma * n ** (alpha - 1))
    assert max(vals) / min(vals) < 1.02


# --------------------------------------------------------------------------- A6
def test_cec_equals_the_fec_bec_combination():
    """CEC (eqs. intro:CEC, intro:CECcoef) evaluated literally as a FEC + b BEC with
    per-cell coefficients agrees with the oracle's singularity-free evaluation, for a
    variable velocity of both signs."""
    n = 64
    rng = np.random.default_rng(7)
    phi = rng.standard_normal(n)
    c = rng.uniform(0.05, 1.0, n) * rng.choice([-1.0, 1.0], n)
    lit = O.scheme_on(phi, c[None], O.CEC_DEF, axis=0)
    assert np.max(np.abs(O.scheme_on(phi, c[None], O.CEC, axis=0) - lit)) < 1e-12
    fec = O.scheme_on(phi, c[None], O.FEC, axis=0)
    bec = O.scheme_on(phi, c[None], O.BEC, axis=0)
    a = (2 - 1 / np.abs(c)) / 3
    assert np.max(np.abs(a * fec + (1 - a) * bec - lit)) < 1e-12


def test_table1_cec_formula_reading():
    """Table 1's CEC row holds with (2U-1)/(6U), not with the printed (1-2U)/(6U)."""
    n, U = 30, 0.37
    phi = np.random.default_rng(8).standard_normal(n)
    c = np.full((1, n), U)
    L = lambda f: O.interp(f, c, +1)  # noqa: E731
    delta = phi - O.interp(L(phi), c, -1)
    reading = L(phi + (1 + U) / (6 * U) * delta) + (2 * U - 1) / (6 * U) * delta
    printed = L(phi + (1 + U) / (6 * U) * delta) + (1 - 2 * U) / (6 * U) * delta
    cec = O.step(phi, c, O.CEC)
    assert np.max(np.abs(cec - reading)) < 1e-14
    assert np.max(np.abs(cec - printed)) > 1e-3


def test_cec_at_zero_velocity_is_identity_there():
    """Where u = 0 the CEC value is the cell's own value (FEC = BEC there)."""
    n = 20
    rng = np.random.default_rng(9)
    phi = rng.standard_normal(n)
    c = rng.uniform(-0.9, 0.9, n)
    c[[3, 11]] = 0.0
    out = O.scheme_on(phi, c[None], O.CEC, axis=0)
    fec = O.scheme_on(phi, c[None], O.FEC, axis=0)
    bec = O.scheme_on(phi, c[None], O.BEC, axis=0)
    assert out[3] == fec[3] == pytest.approx(bec[3], abs=1e-15)
    assert out[3] == phi[3] and out[11] == phi[11]


# --------------------------------------------------------------------------- P9
def cir_matrix(cfield, shape, sign=+1):
    """Matrix of the multilinear CIR operator written from the paper's explicit form
    (eq. CIR2D and its 3D analogue): weights prod_d (1-U_d or U_d) on cells i - s_d e_d."""
    nd = len(shape)
    N = int(np.prod(shape))
    M = np.zeros((N, N))
    for flat in range(N):
        idx = np.unravel_index(flat, shape)        # (z, y, x) order
        pos = idx[::-1]                            # x, y, z
        C = [sign * cfield[d][idx] for d in range(nd)]
        U = [abs(v) for v in C]
        s = [int(np.sign(v)) for v in C]
        for b in range(1 << nd):
            w = 1.0
            q = list(pos)
            for d in range(nd):
                if (b >> d) & 1:
                    w *= U[d]
                    q[d] -= s[d]
                else:
                    w *= 1 - U[d]
            tgt = np.ravel_multi_index(tuple(q[::-1]), shape, mode="wrap")
            M[flat, tgt] += w
    return M


def cir_axis_matrix(ca, shape, axis):
    N = int(np.prod(shape))
    M = np.zeros((N, N))
    nd = len(shape)
    for flat in range(N):
        idx = list(np.unravel_index(flat, shape))
        C = ca[tuple(idx)]
        s = int(np.sign(C))
        q = list(idx)
        q[nd - 1 - axis] -= s
        M[flat, flat] += 1 - abs(C)
        M[flat, np.ravel_multi_index(tuple(q), shape, mode="wrap")] += abs(C)
    return M


def oracle_matrix(fn, shape):
    N = int(np.prod(shape))
    cols = []
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        cols.append(fn(e.reshape(shape)).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("shape", [(5, 4), (4, 3, 5)])
def test_brute_force_matrix_composition(shape):
    """Assemble L from the paper's explicit CIR weights, compose FEC, BEC and the
    split CEC as matrices, and compare with the oracle applied to unit vectors."""
    nd = len(shape)
    N = int(np.prod(shape))
    rng = np.random.default_rng(10 + nd)
    c = rng.uniform(0.05, 0.95, size=(nd,) + shape) * rng.choice([-1.0, 1.0], size=(nd,) + shape)
    I = np.eye(N)
    ML = cir_matrix(c, shape, +1)
    MLm = cir_matrix(c, shape, -1)
    D = I - MLm @ ML                     # Phi - Phi_bar
    mats = {O.CIR: ML, O.FEC: ML + 0.5 * D, O.BEC: ML @ (I + 0.5 * D)}
    # split CEC: per axis a FEC_d + b BEC_d with row coefficients of the output cell
    axis_ops = []
    for d in range(nd):
        MLd = cir_axis_matrix(c[d], shape, d)
        MLdm = cir_axis_matrix(-c[d], shape, d)
        Dd = I - MLdm @ MLd
        U = np.abs(c[d]).ravel()
        a = (2 - 1 / U) / 3
        axis_ops.append(np.diag(a) @ (MLd + 0.5 * Dd) + np.diag(1 - a) @ (MLd @ (I + 0.5 * Dd)))
    for parity in (0, 1):
        order = range(nd) if parity == 0 else reversed(range(nd))
        M = I
        for d in order:
            M = axis_ops[d] @ M
        got = oracle_matrix(lambda f: O.step(f, c, O.CEC, parity), shape)
        assert np.max(np.abs(got - M)) < 1e-12
        assert np.allclose(M.sum(axis=1), 1.0)
    for s, M in mats.items():
        got = oracle_matrix(lambda f: O.step(f, c, s), shape)
        assert np.max(np.abs(got - M)) < 1e-13, NAMES[s]
        assert np.allclose(M.sum(axis=1), 1.0)


# --------------------------------------------------------------------------- sampling
@pytest.mark.parametrize("scheme", ALL)
@pytest.mark.parametrize("shape", [(9, 10, 11), (4, 5, 3), (12, 13)])
def test_sampled_cells_equal_full_step(scheme, shape):
    nd = len(shape)
    rng = np.random.default_rng(11)
    phi = rng.standard_normal(shape)
    c = rng.uniform(-1, 1, size=(nd,) + shape)
    for parity in (0, 1):
        full = O.step(phi, c, scheme, parity)
        cells = np.stack([rng.integers(0, shape[nd - 1 - d], 25) if d < nd else np.zeros(25, int)
                          for d in range(3)], axis=1)
        got = O.sample(phi, c, scheme, parity, cells)
        idx = tuple(cells[:, nd - 1 - a] for a in range(nd))
        assert np.max(np.abs(got - full[idx])) < 1e-14


def test_norms():
    a = np.array([1.0, 2.0, 3.0, 5.0])
    b = np.array([1.0, 2.5, 3.0, 4.0])
    rms, linf, rel = O.norms(a, b)
    assert rms == pytest.approx(math.sqrt((0.25 + 1.0) / 4))
    assert linf == 1.0
    assert rel == pytest.approx(math.sqrt(1.25 / (1 + 6.25 + 9 + 16)))


@pytest.mark.parametrize("U", [0.2, 0.37, 0.8])
def test_bench_table1_coefficients_equal_the_fixture(U):
    """The benchmark's resolution study divides by Table 1's leading
    coefficients, written there as c * u dx^(alpha - 1) for u = 1, dt = U dx;
    they equal the fixture's transcription of Table 1."""
    import bench
    me = GOLD["modified_equation"]
    dx = 1.0 / 256
    dt = U * dx
    for name, (alpha, c) in bench.TABLE1_DECAY.items():
        coeff = ev(me[name][str(alpha)], U=U, u=1.0, dx=dx, dt=dt)
        # the decay rate of exp(i k x) is -Re(C_alpha (i k)^alpha), per k^alpha
        decay = -(coeff * 1j ** alpha).real
        assert decay / dx ** (alpha - 1) == pytest.approx(c(U), rel=1e-12), name
    for name, c in bench.TABLE1_DRIFT.items():
        coeff = ev(me[name]["3"], U=U, u=1.0, dx=dx, dt=dt)
        # the phase drift of exp(i k x) is Im(C_3 (i k)^3) = -C_3 k^3
        assert -coeff / dx ** 2 == pytest.approx(c(U), rel=1e-12), name
