"""The all-cores build of the oracle (-fopenmp over the forward's x-planes)
gives the same bits as the single-threaded build: every point is computed on
its own from the inputs, so sharing the planes among threads changes nothing
but the time it takes."""
import subprocess

import numpy as np
import pytest

import oracle
import workload


@pytest.fixture(scope="module")
def omp():
    try:
        oracle.build(openmp=True)
    except (subprocess.CalledProcessError, OSError) as e:
        pytest.skip(f"gcc cannot build with -fopenmp here: {e}")
    return True


@pytest.mark.parametrize("shape", [(37, 29, 16), (5, 3, 3), (64, 8, 64)])
def test_openmp_build_is_bitwise_the_plain_build(omp, shape):
    winds = workload.winds(*shape, seed=71)
    c = oracle.coefficients(workload.vertical_grid(shape[2]))
    ref = oracle.forward(*winds, c)
    got = oracle.forward(*winds, c, openmp=True)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)


def test_openmp_build_respects_plane_range(omp):
    shape = (40, 12, 24)
    winds = workload.winds(*shape, seed=72)
    c = oracle.coefficients(workload.vertical_grid(shape[2]))
    ref = oracle.forward(*winds, c, i_range=(3, 31))
    got = oracle.forward(*winds, c, i_range=(3, 31), openmp=True)
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
        assert not g[:3].any() and not g[31:].any()


def test_thread_counts(omp):
    assert oracle.threads() == 1
    assert oracle.threads(openmp=True) >= 1
