"""Degenerate cases of the method on the GPU path, each against the oracle or an exact value:
a zero state, a decoupled species pair (b_ij = 0), one radial node with one direction, a
user-set truncation radius, identical species of equal mass, and a large mass ratio."""

import numpy as np
import pytest

from gpu_helpers import check, gpu_collision, oracle_collision
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    dgfs.load()


def _inputs(N, L, masses, B, seed):
    w = synth.Workload("edge", B, N, L, tuple(masses), 0.7, 1.0, 6, 3, "bimaxwellian", 0.05, seed)
    return synth.batch_distribution(w)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("alpha", [1.0, 1.4])
def test_zero_state_gives_exactly_zero(precision, alpha):
    """Q is bilinear in (f_i, f_j): f = 0 gives Q = 0 exactly, in every precision."""
    f = np.zeros((2, 2, 8, 8, 8))
    Q = gpu_collision(f, N=8, L=4.0, masses=(1.0, 2.0), omega=0.7, alpha=alpha, M=6, N_rho=3,
                      precision=precision)
    assert not np.any(Q)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_decoupled_pair_is_exactly_zero(precision):
    """b_12 = b_21 = 0: the kernel vanishes for the cross pair, so Q_12 = Q_21 = 0 exactly,
    while the self pairs match the oracle."""
    b = np.array([[0.3, 0.0], [0.0, 0.2]])
    kw = dict(N=8, L=4.0, masses=(1.0, 2.0), omega=0.7, M=6, N_rho=3, b_override=b)
    f = _inputs(8, 4.0, (1.0, 2.0), 2, seed=31)
    Q = gpu_collision(f, precision=precision, **kw)
    ref = oracle_collision(f, **kw)
    assert not np.any(Q[:, 0, 1]) and not np.any(Q[:, 1, 0])
    assert not np.any(ref[:, 0, 1]) and not np.any(ref[:, 1, 0])
    for i in range(2):
        own = (slice(None), slice(i, i + 1), slice(i, i + 1))
        assert check(Q[own], ref[own], precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("alpha", [1.0, 1.4])
def test_one_radial_node_one_direction(precision, alpha):
    """N_rho = 1 and a one-point sphere rule (no antipode): the smallest quadrature."""
    sigma = np.array([[0.0, 0.6, 0.8]])
    kw = dict(N=8, L=4.0, masses=(1.0, 2.0), omega=0.7, alpha=alpha, N_rho=1, sigma=sigma,
              w_sigma=np.array([4 * np.pi]))
    f = _inputs(8, 4.0, (1.0, 2.0), 2, seed=32)
    assert check(gpu_collision(f, precision=precision, **kw), oracle_collision(f, **kw), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_user_truncation_radius(precision):
    kw = dict(N=12, L=5.0, masses=(1.0, 3.0), omega=0.6, M=6, N_rho=3, R=2.5)
    f = _inputs(12, 5.0, (1.0, 3.0), 2, seed=33)
    assert check(gpu_collision(f, precision=precision, **kw), oracle_collision(f, **kw), precision)


def test_identical_species_give_equal_operators():
    """Two species of equal mass in the same state: all four operators are the same function
    (the self pairs run halved, the cross pair over all directions, so they agree to
    rounding), and they match the single-species operator."""
    f1 = _inputs(8, 4.0, (1.0, 1.0), 2, seed=34)[:, :1]
    f = np.concatenate([f1, f1], axis=1)
    Q = gpu_collision(f, N=8, L=4.0, masses=(1.0, 1.0), omega=0.7, M=12, N_rho=3, precision="fp64")
    Q1 = gpu_collision(f1, N=8, L=4.0, masses=(1.0,), omega=0.7, M=12, N_rho=3, precision="fp64")
    scale = np.max(np.abs(Q1))
    for i in range(2):
        for j in range(2):
            assert np.max(np.abs(Q[:, i, j] - Q1[:, 0, 0])) < 1e-12 * scale


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_large_mass_ratio(precision):
    """m_2/m_1 = 25: the domain rule leaves a small support radius; still parity."""
    kw = dict(N=12, L=5.0, masses=(1.0, 25.0), omega=0.8, M=6, N_rho=3)
    f = _inputs(12, 5.0, (1.0, 25.0), 2, seed=35)
    assert check(gpu_collision(f, precision=precision, **kw), oracle_collision(f, **kw), precision)
