"""The learned corrector: feature extraction, tensor-core MLP inference, training
and the plain-scheme check with fallback.  The corrector's output has no oracle
(the paper has no such scheme), so its arithmetic is checked against a plain
PyTorch float64 evaluation of the same network on the same BF16-rounded
operands, and its accuracy is judged against the plain CEC step."""
import math

import numpy as np
import pytest
import torch

from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
NIN, NH = 67, 64


def hash32(x):
    x = np.uint32(x)
    with np.errstate(over="ignore"):
        x ^= x >> np.uint32(16)
        x = np.uint32((int(x) * 0x7FEB352D) & 0xFFFFFFFF)
        x ^= x >> np.uint32(15)
        x = np.uint32((int(x) * 0x846CA68B) & 0xFFFFFFFF)
        x ^= x >> np.uint32(16)
    return int(x)


def sample_cell(seed, j, ncell):
    s = (seed ^ (seed >> 32)) & 0xFFFFFFFF
    h = hash32((s * 0x9E3779B9 + j) & 0xFFFFFFFF)
    return (h * hash32(h ^ 0x5BD1E995)) % ncell


def ref_features(phi, vel, sp, dt, x, y, z):
    """The corrector's inputs of one cell, float64 from the float32 fields."""
    nz, ny, nx = phi.shape
    C = [np.float32(vel[d, z, y, x]) * np.float32(dt / sp[d]) for d in range(3)]
    I = [x, y, z]
    Xd = [np.float32(np.float32(I[d]) - C[d]) for d in range(3)]
    b = [min(int(math.floor(Xd[d])), I[d]) for d in range(3)]
    f = [float(Xd[d]) - b[d] for d in range(3)]
    v = np.empty(64)
    for c in range(4):
        for bb in range(4):
            for a in range(4):
                v[a + 4 * bb + 16 * c] = phi[(b[2] - 1 + c) % nz, (b[1] - 1 + bb) % ny, (b[0] - 1 + a) % nx]
    inner = v.reshape(4, 4, 4)[1:3, 1:3, 1:3]      # [z][y][x]
    wx = np.array([1 - f[0], f[0]])
    wy = np.array([1 - f[1], f[1]])
    wz = np.array([1 - f[2], f[2]])
    m = float(np.einsum("zyx,z,y,x->", inner, wz, wy, wx))
    s = max(np.abs(v - m).max(), 1e-30)
    feat = np.concatenate([(v - m) / s, np.array(f) - 0.5])
    return feat, m, s


def bf16(a):
    return torch.tensor(a, dtype=torch.float64).to(torch.bfloat16).to(torch.float64).numpy()


def ref_mlp(params, feat):
    """Same network, float64 arithmetic on the BF16 operands the kernel uses."""
    o = 0
    W1 = params[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = params[o:o + NH]; o += NH
    W2 = params[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = params[o:o + NH]; o += NH
    w3 = params[o:o + NH]; o += NH
    b3 = params[o]
    h1 = np.maximum(bf16(W1) @ bf16(feat) + b1, 0.0)
    h2 = np.maximum(bf16(W2) @ bf16(h1) + b2, 0.0)
    return float(h2 @ w3 + b3)


def small_case(shape=(6, 8, 64), seed=3, cmax=0.9):
    rng = np.random.default_rng(seed)
    phi = W.random_modes(shape, W.draw_modes(3, 8, 3, seed=seed), dtype=torch.float32)
    sp = [0.1, 0.2, 0.15]
    dt = 0.05
    C = rng.uniform(-cmax, cmax, size=(3,) + shape)
    vel = torch.from_numpy(np.stack([C[d] * sp[d] / dt for d in range(3)])).float()
    return phi, vel, sp, dt


def test_training_rows_match_reference_features():
    phi, vel, sp, dt = small_case()
    shape = phi.shape
    dims = [shape[2], shape[1], shape[0]]
    p, v = phi.to(DEV), vel.to(DEV)
    target = sl.advect(p, v, dt, sp, "CEC", 0)
    c = sl.sl_corrector_create(1)
    try:
        seed = 12345
        sl.sl_corrector_add_samples(c, p, target, v, dims, sp, dt, 200, seed)
        torch.cuda.synchronize()
        rows = sl.sl_corrector_get_rows(c, 0, 200)
    finally:
        sl.sl_corrector_destroy(c)
    ph, ve, tg = phi.numpy(), vel.numpy(), target.cpu().numpy()
    ncell = phi.numel()
    for j in range(200):
        cell = sample_cell(seed, j, ncell)
        z, y, x = cell // (shape[1] * shape[2]), (cell // shape[2]) % shape[1], cell % shape[2]
        feat, m, s = ref_features(ph, ve, sp, dt, x, y, z)
        assert np.allclose(rows[j, :NIN], feat, atol=2e-5), j
        assert rows[j, 67] == pytest.approx((tg[z, y, x] - m) / s, abs=2e-4)


def test_tensor_core_inference_matches_reference_mlp():
    phi, vel, sp, dt = small_case(seed=4)
    shape = phi.shape
    dims = [shape[2], shape[1], shape[0]]
    rng = np.random.default_rng(7)
    c = sl.sl_corrector_create(2)
    try:
        params = (rng.standard_normal(sl.sl_corrector_param_count()) * 0.2).astype(np.float32)
        sl.sl_corrector_set_params(c, params)
        out = torch.empty(shape, device=DEV)
        used, _ = sl.sl_advect_learned(c, out, phi.to(DEV), vel.to(DEV), 3, dims, sp, dt)
        torch.cuda.synchronize()
        assert used == 0
    finally:
        sl.sl_corrector_destroy(c)
    got = out.cpu().numpy()
    ph, ve = phi.numpy(), vel.numpy()
    p64 = params.astype(np.float64)
    errs = []
    rng2 = np.random.default_rng(8)
    cells = [(int(rng2.integers(shape[2])), int(rng2.integers(shape[1])), int(rng2.integers(shape[0])))
             for _ in range(300)]
    for x, y, z in cells:
        feat, m, s = ref_features(ph, ve, sp, dt, x, y, z)
        yv = ref_mlp(p64, feat)
        errs.append(abs(got[z, y, x] - (m + s * yv)) / (s * (1.0 + abs(yv))))
    errs = np.array(errs)
    assert np.quantile(errs, 0.99) < 5e-3 and errs.max() < 5e-2, (np.median(errs), errs.max())


def test_training_reduces_loss_and_learned_step_is_checked():
    shape = (32, 32, 64)
    dims = [64, 32, 32]
    sp = [2 * math.pi / n for n in dims]
    phi = W.random_modes(shape, W.draw_modes(3, 16, 4, seed=9), device=DEV, dtype=torch.float32)
    vel = W.abc_velocity(shape, device=DEV, dtype=torch.float32)
    dt = 0.8 * min(sp) / 2.0
    c = sl.sl_corrector_create(3)
    try:
        cur = phi
        for k in range(4):
            nxt = sl.advect(cur, vel, dt, sp, "CEC", 0)
            sl.sl_corrector_add_samples(c, cur, nxt, vel, dims, sp, dt, 50000, seed=100 + k)
            cur = nxt
        first = sl.sl_corrector_train(c, 1, 2048, 2e-3, seed=1)
        last = sl.sl_corrector_train(c, 600, 2048, 2e-3, seed=2)
        assert last < first / 5, (first, last)
        out = torch.empty_like(phi)
        used, errs = sl.sl_advect_learned(c, out, cur, vel, 3, dims, sp, dt, 0, check=1, fallback_ratio=1e9)
        assert used == 0 and np.isfinite(errs[0]) and np.isfinite(errs[1])
        # with a zero tolerance the check must fall back and hand out the plain step
        used, errs = sl.sl_advect_learned(c, out, cur, vel, 3, dims, sp, dt, 0, check=1, fallback_ratio=0.0)
        assert used == 1
        assert torch.equal(out, sl.advect(cur, vel, dt, sp, "CEC", 0))
        # later unchecked steps stay on the plain scheme until reset
        used, _ = sl.sl_advect_learned(c, out, cur, vel, 3, dims, sp, dt, 1)
        assert used == 1 and torch.equal(out, sl.advect(cur, vel, dt, sp, "CEC", 1))
        sl.sl_corrector_reset(c)
        used, _ = sl.sl_advect_learned(c, out, cur, vel, 3, dims, sp, dt, 0)
        assert used == 0
    finally:
        sl.sl_corrector_destroy(c)


def test_learned_rejects_unsupported_grids():
    c = sl.sl_corrector_create(4)
    try:
        a = torch.zeros(8, 8, 8, device=DEV)
        v = torch.zeros(3, 8, 8, 8, device=DEV)
        with pytest.raises(sl.SLError) as e:
            sl.sl_advect_learned(c, torch.empty_like(a), a, v, 3, [8, 8, 8], [1, 1, 1], 0.1)
        assert e.value.code == -6
        # a supported shape whose input does not start on a 16-byte boundary
        base = torch.zeros(3 * 4 * 32 + 1, device=DEV)
        shifted = base[1:].view(3, 4, 32)
        v2 = torch.zeros(3, 3, 4, 32, device=DEV)
        with pytest.raises(sl.SLError) as e:
            sl.sl_advect_learned(c, torch.empty(3, 4, 32, device=DEV), shifted, v2, 3, [32, 4, 3], [1, 1, 1], 0.1)
        assert e.value.code == -6 and "aligned" in str(e.value)
    finally:
        sl.sl_corrector_destroy(c)


def _trained_corrector(shape=(64, 64, 64), iters=400, seed=5):
    """A corrector trained on pairs of plain CEC steps of an ABC / random-mode field."""
    dims = [shape[2], shape[1], shape[0]]
    sp = [2 * math.pi / n for n in dims]
    vel = W.abc_velocity(shape, device=DEV, dtype=torch.float32)
    dt = 0.8 * min(sp) / 2.0
    c = sl.sl_corrector_create(seed)
    cur = W.random_modes(shape, W.draw_modes(3, 16, 4, seed=seed), device=DEV, dtype=torch.float32)
    for k in range(3):
        nxt = sl.advect(cur, vel, dt, sp, "CEC", 0)
        sl.sl_corrector_add_samples(c, cur, nxt, vel, dims, sp, dt, 60000, seed=200 + k)
        cur = sl.advect(cur, vel, dt, sp, "CEC", k)
    sl.sl_corrector_train(c, iters, 2048, 2e-3, seed=3)
    return c, cur, vel, dims, sp, dt


def test_learned_step_error_is_measured_against_the_oracle():
    """The check judges the learned step by its distance from the plain
    third-order step computed on the GPU.  On sampled cells, the FP64 oracle's
    step gives the same distance to within the GPU step's own error against the
    oracle (FP32 rounding), so the check is a judgement against the oracle; the
    two errors are reported beside each other."""
    from gpu_helpers import oracle_at_cells, rel_l2, sample_cells
    c, cur, vel, dims, sp, dt = _trained_corrector()
    try:
        shape = tuple(cur.shape)
        learned = torch.empty_like(cur)
        used, errs = sl.sl_advect_learned(c, learned, cur, vel, 3, dims, sp, dt, 0, check=0)
        assert used == 0
        plain = sl.advect(cur, vel, dt, sp, "CEC", 0)
        cells = sample_cells(shape, 800, seed=7)
        ref = oracle_at_cells(cur, vel, sp, dt, "CEC", 0, cells)
        at = lambda t: t[cells[:, 2], cells[:, 1], cells[:, 0]].cpu().double().numpy()
        plain_vs_oracle = rel_l2(at(plain), ref)
        learned_vs_oracle = rel_l2(at(learned), ref)
        learned_vs_plain = rel_l2(at(learned), at(plain))
        print(f"learned vs oracle {learned_vs_oracle:.3e}, plain CEC vs oracle {plain_vs_oracle:.3e}")
        assert plain_vs_oracle <= 1e-5
        assert abs(learned_vs_oracle - learned_vs_plain) <= plain_vs_oracle + 1e-7
        # the checked step's learned error (whole field, against the GPU step)
        used, errs = sl.sl_advect_learned(c, torch.empty_like(cur), cur, vel, 3, dims, sp, dt, 0, check=1,
                                          fallback_ratio=1e9)
        assert used == 0 and abs(errs[0] - learned_vs_plain) <= 0.5 * learned_vs_plain
    finally:
        sl.sl_corrector_destroy(c)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_corrupted_weights_fall_back_to_the_plain_step(bad):
    """Host-side fault injection: a non-finite weight written through
    sl_corrector_set_params makes the next checked step hand out the plain CEC
    step and keeps the corrector on the plain scheme until reset."""
    c, cur, vel, dims, sp, dt = _trained_corrector(iters=50)
    try:
        params = np.empty(sl.sl_corrector_param_count(), dtype=np.float32)
        params[:] = sl.sl_corrector_get_params(c)
        params[5] = bad                                   # one entry of W1
        sl.sl_corrector_set_params(c, params)
        out = torch.empty_like(cur)
        used, errs = sl.sl_advect_learned(c, out, cur, vel, 3, dims, sp, dt, 1, check=1, fallback_ratio=2.0)
        assert used == 1
        assert torch.equal(out, sl.advect(cur, vel, dt, sp, "CEC", 1))
        used, _ = sl.sl_advect_learned(c, out, cur, vel, 3, dims, sp, dt, 0)
        assert used == 1 and torch.equal(out, sl.advect(cur, vel, dt, sp, "CEC", 0))
        assert torch.isfinite(out).all()
    finally:
        sl.sl_corrector_destroy(c)
