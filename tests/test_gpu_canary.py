"""Out-of-bounds writes would corrupt what lies next to the output: every
kernel family writes its step into the middle of a buffer whose padding holds
a canary bit pattern (a NaN payload no kernel produces), and every padding word
must come back unchanged.  The inputs sit in canary-padded buffers too.
(compute-sanitizer is closed on this machine; this and the bounded parity cases
stand in for it.)"""
import math

import pytest
import torch

from paper_1606_06117_gb300 import _lib as sl
from paper_1606_06117_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = "cuda"
PAD = 4096                      # elements of padding on each side (16 KB in FP32)
CANARY32 = 0x7FBADBAD           # quiet-NaN payloads
CANARY64 = 0x7FF8BADBADBADBAD


def padded(t):
    """A copy of t inside a canary-padded buffer; returns (buffer, view)."""
    n = t.numel()
    if t.dtype == torch.float64:
        buf = torch.full((n + 2 * PAD,), CANARY64, dtype=torch.int64, device=DEV).view(torch.float64)
    else:
        buf = torch.full((n + 2 * PAD,), CANARY32, dtype=torch.int32, device=DEV).view(torch.float32)
    view = buf[PAD:PAD + n].view(t.shape)
    view.copy_(t)
    return buf, view


def canaries_intact(buf):
    torch.cuda.synchronize()
    ints = buf.view(torch.int64 if buf.dtype == torch.float64 else torch.int32)
    want = CANARY64 if buf.dtype == torch.float64 else CANARY32
    return bool((ints[:PAD] == want).all()) and bool((ints[-PAD:] == want).all())


def smooth(shape, dtype=torch.float32, cfl=0.9):
    nz, ny, nx = shape
    phi = W.random_modes(shape, W.draw_modes(3, 8, 3, seed=sum(shape)), device=DEV, dtype=dtype)
    vel = W.abc_velocity(shape, device=DEV, dtype=dtype)
    sp = [2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz]
    return phi, vel, sp, cfl * min(sp) / 2.0


# (torch shape, schemes, dtype): the fast CEC kernels, the generic split and
# unsplit kernels, the four-cell CIR kernel, FP64 and FP32 with FP64 delta
CASES = [((64, 64, 64), ["CEC"], torch.float32, False), ((20, 36, 40), ["CEC", "CIR", "FEC", "BEC"], torch.float32, False),
         ((23, 48, 100), ["CIR", "FEC", "BEC"], torch.float32, False), ((9, 10, 12), ["CIR", "BEC", "CEC"], torch.float64, False),
         ((16, 32, 64), ["CEC"], torch.float32, True), ((1, 40, 52), ["CIR", "CEC"], torch.float32, False)]


@pytest.mark.parametrize("shape,schemes,dtype,d64", CASES)
def test_steps_write_nothing_outside_their_output(shape, schemes, dtype, d64):
    phi, vel, sp, dt = smooth(shape, dtype)
    if shape[0] == 1:
        phi, vel, sp = phi[0], vel[:2, 0], sp[:2]
    ibuf, pin = padded(phi)
    vbuf, vin = padded(vel)
    for scheme in schemes:
        for parity in (0, 1):
            obuf, out = padded(torch.zeros_like(phi))
            sl.advect(pin, vin, dt, sp, scheme, parity, out=out, delta64=d64)
            assert canaries_intact(obuf), (scheme, shape, parity)
            assert torch.isfinite(out).all()
    assert canaries_intact(ibuf) and canaries_intact(vbuf)
    assert sl.sl_device_status() == 0


def test_wide_step_writes_nothing_outside_output_or_workspace():
    shape = (16, 24, 32)
    phi, vel, sp, dt = smooth(shape, cfl=3.0)
    ibuf, pin = padded(phi)
    vbuf, vin = padded(vel)
    for scheme in ("CIR", "FEC", "BEC", "CEC"):
        need = sl.sl_advect_wide_workspace(3, list(shape[::-1]), sl.SCHEMES[scheme], sl.F32)
        wbuf = torch.full((need // 4 + 2 * PAD + 64,), CANARY32, dtype=torch.int32, device=DEV)
        base = wbuf.data_ptr() + 4 * PAD
        base += (-base) % 256
        off = (base - wbuf.data_ptr()) // 4
        obuf, out = padded(torch.zeros_like(phi))
        sl.sl_advect_wide(out, pin, vin, 3, list(shape[::-1]), sp, dt, sl.SCHEMES[scheme], sl.F32, 0, base, need)
        torch.cuda.synchronize()
        assert canaries_intact(obuf), scheme
        assert bool((wbuf[:off] == CANARY32).all()) and bool((wbuf[off + need // 4:] == CANARY32).all()), scheme
    assert canaries_intact(ibuf) and canaries_intact(vbuf)


def test_multi_field_and_batched_steps_write_nothing_outside_their_outputs():
    shape = (32, 64, 64)
    phi, vel, sp, dt = smooth(shape)
    ins = [padded(phi * (k + 1)) for k in range(3)]
    outs = [padded(torch.zeros_like(phi)) for _ in range(3)]
    sl.sl_advect_multi([o for _, o in outs], [i for _, i in ins], vel, 3, [64, 64, 32], sp, dt, sl.CEC, sl.F32, 1)
    assert all(canaries_intact(b) for b, _ in outs) and all(canaries_intact(b) for b, _ in ins)
    recs, keep = [], []
    for shp in ((32, 64, 64), (20, 36, 40)):
        p, v, s, d = smooth(shp)
        (ab, a), (bb, b) = padded(p), padded(torch.zeros_like(p))
        keep.append((ab, a, bb, b, v))
        recs.append(sl.Instance(a.data_ptr(), b.data_ptr(), v.data_ptr(), tuple(shp[::-1]), tuple(s), d))
    h = sl.sl_batch_create(recs)
    try:
        for k in range(2):
            sl.sl_batch_step(h, k)
    finally:
        sl.sl_batch_destroy(h)
    assert all(canaries_intact(ab) and canaries_intact(bb) for ab, _, bb, _, _ in keep)
    assert sl.sl_device_status() == 0


def test_learned_step_writes_nothing_outside_its_output():
    shape = (32, 32, 64)
    phi, vel, sp, dt = smooth(shape)
    ibuf, pin = padded(phi)
    c = sl.sl_corrector_create(3)
    try:
        for check in (0, 1):
            obuf, out = padded(torch.zeros_like(phi))
            sl.sl_advect_learned(c, out, pin, vel, 3, [64, 32, 32], sp, dt, 0, check=check)
            assert canaries_intact(obuf), check
    finally:
        sl.sl_corrector_destroy(c)
    assert canaries_intact(ibuf)
