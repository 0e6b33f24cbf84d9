"""The C ABI used from plain C99: tests/abi_c/forward_host.c includes only
include/advect.h and links only the library.

CPU: the program compiles warning-free as C99 and links against the built
library.  GPU: it runs the forward pass from host buffers and its output
matches the oracle on the same inputs (FP64 bar, 1e-12 normwise).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import workload
from paper_2010_01545_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "abi_c", "forward_host.c")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


def _compile(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib = build.build()
    exe = tmp_path / "forward_host"
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-O2", "-I", INCLUDE, SRC, "-o", str(exe),
           "-L", libdir, "-ladvect", f"-Wl,-rpath,{libdir}", "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_c_program_compiles_and_links(tmp_path):
    assert os.path.exists(_compile(tmp_path))


def _pattern(shape):
    nx, ny, nz = shape
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    return [8.0 * np.sin(0.37 * i + 0.23 * j + 0.11 * k + 1.3 * f) + 0.5 * f for f in range(3)]


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(16, 12, 8), (33, 17, 64), (1, 1, 3)])
def test_c_program_forward_matches_oracle(tmp_path, shape):
    exe = _compile(tmp_path)
    out = tmp_path / "s.bin"
    r = subprocess.run([str(exe), *map(str, shape), str(out)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = np.fromfile(out, dtype=np.float64).reshape(3, *shape)
    nz = shape[2]
    z = 10.0 * np.arange(nz)
    grid = workload.custom_grid(z, z - 5.0, np.ones(nz), np.ones(nz), 50.0, 50.0)
    ref = oracle.forward(*_pattern(shape), oracle.coefficients(grid))
    for g, rr in zip(got, ref):
        assert np.max(np.abs(g - rr)) <= 1e-12 * max(np.max(np.abs(rr)), 1e-300)
