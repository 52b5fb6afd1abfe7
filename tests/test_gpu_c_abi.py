"""libsl from plain C: tests/c_abi_step.c, compiled against include/sl.h and
linked with libsl.so, runs two CEC steps through device buffers and through
host buffers (equal bit for bit, checked in C).  Its result must equal the
Python binding's steps on the same inputs bit for bit and the FP64 oracle
within the FP32 bar."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import torch

from gpu_helpers import assert_parity, oracle_step
from paper_1606_06117_gb300 import _lib as sl

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
NX, NY, NZ = 64, 64, 32


def cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def seeded_inputs():
    """The C program's inputs: a 32-bit LCG mapped to [-1, 1) in float32, and
    constant Courant numbers (0.3, -0.2, 0.45) on spacings (0.5, 0.25, 2)."""
    n = NX * NY * NZ
    s = 12345
    phi = np.empty(n, dtype=np.float32)
    for i in range(n):
        s = (s * 1664525 + 1013904223) & 0xFFFFFFFF
        phi[i] = np.float32((s >> 8) * (1.0 / 16777216.0)) * np.float32(2.0) - np.float32(1.0)
    sp, dt = [0.5, 0.25, 2.0], 0.1
    vel = np.stack([np.full(n, np.float32(c * h / dt), dtype=np.float32)
                    for c, h in zip((0.3, -0.2, 0.45), sp)])
    return phi.reshape(NZ, NY, NX), vel.reshape(3, NZ, NY, NX), sp, dt


def test_c_program_steps_equal_the_binding_and_the_oracle(tmp_path):
    sl.load()
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    cuda = cuda_home()
    libdir = os.path.dirname(sl.library_path())
    exe = tmp_path / "c_abi_step"
    cmd = [gcc, "-O1", os.path.join(HERE, "c_abi_step.c"), "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), "-L", libdir, "-lsl", "-L", os.path.join(cuda, "lib64"), "-lcudart",
           f"-Wl,-rpath,{libdir}", "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = tmp_path / "out.bin"
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join([libdir, os.path.join(cuda, "lib64"), env.get("LD_LIBRARY_PATH", "")])
    r = subprocess.run([str(exe), str(out)], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and "C_ABI_OK" in r.stdout, (r.returncode, r.stdout, r.stderr)
    got = np.fromfile(out, dtype=np.float32).reshape(NZ, NY, NX)

    phi, vel, sp, dt = seeded_inputs()
    a = torch.from_numpy(phi).cuda()
    v = torch.from_numpy(vel).cuda()
    b = sl.advect(sl.advect(a, v, dt, sp, "CEC", 0), v, dt, sp, "CEC", 1)
    assert np.array_equal(b.cpu().numpy(), got)
    ref = oracle_step(torch.from_numpy(oracle_step(torch.from_numpy(phi), torch.from_numpy(vel), sp, dt, "CEC", 0)),
                      torch.from_numpy(vel), sp, dt, "CEC", 1)
    assert_parity(got, ref, "f32", "C program, two CEC steps", allowance=2.0)
