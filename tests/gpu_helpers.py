"""Shared helpers of the GPU parity tests: seeded cases, oracle comparison and
periodic windows around sampled cells (so that full-size grids can be checked
cell by cell without copying them to the host)."""
import numpy as np
import torch

from oracle import oracle as O

TOL = {"f32": 1e-5, "f32_d64": 1e-5, "f64": 1e-12}
# cell-by-cell bound, as a fraction of max |oracle|
EW = {"f32": 1e-5, "f32_d64": 1e-5, "f64": 1e-12}
TORCH_DT = {"f32": torch.float32, "f32_d64": torch.float32, "f64": torch.float64}


def random_case(shape, seed, cmax=0.95, dtype="f32", spacing=None, dt=0.1):
    """Random field and per-cell random velocity with |C| <= cmax (sign flips
    from cell to cell exercise every upwind branch)."""
    nd = len(shape)
    rng = np.random.default_rng(seed)
    spacing = list(spacing or [0.5, 0.25, 2.0][:nd])
    phi = rng.standard_normal(shape)
    C = rng.uniform(-cmax, cmax, size=(nd,) + shape)
    vel = np.stack([C[d] * spacing[d] / dt for d in range(nd)])
    t = TORCH_DT[dtype]
    return torch.from_numpy(phi).to(t), torch.from_numpy(vel).to(t), spacing, dt


def courant(vel, spacing, dt):
    """Courant numbers of the exact values the GPU receives, in float64."""
    v = vel.detach().cpu().double().numpy()
    return np.stack([v[d] * (dt / spacing[d]) for d in range(v.shape[0])])


def oracle_step(phi, vel, spacing, dt, scheme, parity):
    return O.step(phi.detach().cpu().double().numpy(), courant(vel, spacing, dt), O.SCHEMES[scheme], parity)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def assert_parity(got, ref, dtype, what="", allowance=1.0):
    """A GPU result against the oracle's: relative L2 <= TOL[dtype] and, cell by
    cell, |got - ref| <= EW[dtype] * max |ref|, both times `allowance` (multi-step
    runs).  The cell-by-cell bound catches a defect confined to a few cells (a seam
    or halo error) that a global norm would average away; a failure names the worst
    cell (its index in `ref`'s shape) and both values."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    err = rel_l2(got, ref)
    diff = np.abs(got - ref)
    if not np.all(np.isfinite(diff)):
        k = int(np.argmax(~np.isfinite(diff).ravel()))
        raise AssertionError(f"{what}: non-finite result at {np.unravel_index(k, diff.shape)}")
    scale = max(float(np.abs(ref).max()), 1e-300)
    k = int(np.argmax(diff))
    worst = float(diff.ravel()[k]) / scale
    ok = err <= allowance * TOL[dtype] and worst <= allowance * EW[dtype]
    assert ok, (f"{what}: relative L2 {err:.3e} (bar {allowance * TOL[dtype]:.1e}); worst cell "
                f"{np.unravel_index(k, diff.shape)} off by {worst:.3e} of max|oracle| (bar "
                f"{allowance * EW[dtype]:.1e}): GPU {got.ravel()[k]!r}, oracle {ref.ravel()[k]!r}")
    return err, worst


def sample_cells(shape, n, seed):
    """n random cells as (x, y, z) rows, plus every corner-ish cell near the wrap."""
    rng = np.random.default_rng(seed)
    dims = list(shape)[::-1] + [1] * (3 - len(shape))
    cells = np.stack([rng.integers(0, dims[d], n) for d in range(3)], axis=1)
    edge = np.array([[0, 0, 0], [dims[0] - 1, dims[1] - 1, dims[2] - 1], [0, dims[1] - 1, 0],
                     [dims[0] - 1, 0, dims[2] - 1]])
    return np.concatenate([cells, edge])


def windows(t, cells, r=3):
    """(n, 2r+1, 2r+1, 2r+1) periodic windows of a (nz, ny, nx) tensor (or a
    stack of them, leading dim kept) centred on cells, gathered on the device."""
    lead = t.shape[:-3]
    nz, ny, nx = t.shape[-3:]
    c = torch.as_tensor(cells, device=t.device, dtype=torch.int64)
    off = torch.arange(-r, r + 1, device=t.device)
    zi = (c[:, 2, None] + off[None]) % nz
    yi = (c[:, 1, None] + off[None]) % ny
    xi = (c[:, 0, None] + off[None]) % nx
    flat = t.reshape(*lead, -1)
    idx = (zi[:, :, None, None] * ny + yi[:, None, :, None]) * nx + xi[:, None, None, :]
    out = flat[..., idx.reshape(-1)].reshape(*lead, len(cells), 2 * r + 1, 2 * r + 1, 2 * r + 1)
    return out


def oracle_at_cells(phi, vel, spacing, dt, scheme, parity, cells):
    """The oracle's step at the given cells, evaluated on periodic 7^3 windows."""
    wp = windows(phi, cells).cpu().double().numpy()
    wv = windows(vel, cells).cpu().double().numpy()          # (3, n, 7, 7, 7)
    out = np.empty(len(cells))
    for i in range(len(cells)):
        c = np.stack([wv[d, i] * (dt / spacing[d]) for d in range(3)])
        out[i] = O.step(wp[i], c, O.SCHEMES[scheme], parity)[3, 3, 3]
    return out
