"""VSS kernel (alpha != 1): sigma-dependent complex gain weights F(k, rho, sigma) built on the
device by the Gauss-Jacobi x J0 form of Eq. GG, one forward transform per (rho, sigma)
entry.  Parity with the oracle (FP64 1e-11 per pair, FP32 1e-5 per node)."""

import numpy as np
import pytest

from gpu_helpers import check, gpu_collision, oracle_collision
from oracle import quadrature
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    dgfs.load()


def _inputs(N, L, masses, B, seed):
    w = synth.Workload("vss", B, N, L, tuple(masses), 0.74, 1.4, 6, 4, "skewed", 0.0, seed)
    return synth.batch_distribution(w)


CASES = {
    "n8_two_species_octahedron": dict(N=8, L=4.0, masses=(1.0, 2.0), omega=0.74, alpha=1.4, M=6, N_rho=3, B=3),
    "n12_three_species_icosahedron": dict(N=12, L=5.0, masses=(1.0, 1.5, 2.6), omega=0.74, alpha=1.4, M=12, N_rho=3, B=2),
    "n16_m32_design": dict(N=16, L=6.0, masses=(1.0, 2.6), omega=0.74, alpha=1.4, M=32, N_rho=2, B=1),
    "n12_alpha2": dict(N=12, L=5.0, masses=(1.0, 3.0), omega=0.6, alpha=2.0, M=6, N_rho=3, B=2),
    # N = 32 runs the FP32 tensor-memory shape (8-CTA clusters, dynamic pencil passes)
    "n32_two_species": dict(N=32, L=7.0, masses=(1.0, 2.1), omega=0.81, alpha=1.4, M=6, N_rho=2, B=2),
}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_vss_parity_with_oracle(name, precision):
    kw = dict(CASES[name])
    B = kw.pop("B")
    f = _inputs(kw["N"], kw["L"], kw["masses"], B, seed=70 + kw["N"])
    Q = gpu_collision(f, precision=precision, **kw)
    ref = oracle_collision(f, **kw)
    assert check(Q, ref, precision)


_N48 = {}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vss_n48_parity_with_oracle(precision):
    """One node of the N = 48 VSS grid (L = 8, masses 1 : 2.6, alpha = 1.4) against the
    oracle.  With N_rho = 2 the outer radial node reaches a = pi rho c_j |k| / L ~ 51 at the
    corner modes, where the t rule of F must be converged (the oracle doubles its rule until
    it is; the plan sizes its rule from the largest argument).  The oracle's gain tables take
    about a minute here, so its result is shared by both precisions."""
    kw = dict(N=48, L=8.0, masses=(1.0, 2.6), omega=0.74, alpha=1.4, M=6, N_rho=2)
    if "f" not in _N48:
        _N48["f"] = _inputs(48, 8.0, (1.0, 2.6), 1, seed=148)
        _N48["ref"] = oracle_collision(_N48["f"], **kw)
    Q = gpu_collision(_N48["f"], precision=precision, **kw)
    assert check(Q, _N48["ref"], precision)


def test_vss_mixed_alpha_per_pair():
    """alpha may differ per pair; alpha_ij = 1 pairs then go through the same sigma-dependent
    path and must agree with the VHS closed form the oracle uses for them."""
    alpha = np.array([[1.0, 1.5], [1.5, 1.2]])
    kw = dict(N=8, L=4.0, masses=(1.0, 2.0), omega=0.7, alpha=alpha, M=6, N_rho=3)
    f = _inputs(8, 4.0, (1.0, 2.0), 2, seed=91)
    assert check(gpu_collision(f, precision="fp64", **kw), oracle_collision(f, **kw), "fp64")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vss_non_antipodal_rule(precision):
    """A rule without antipodes: one table slot per direction, no conjugate reads."""
    rng = np.random.default_rng(12)
    sigma = rng.normal(size=(5, 3))
    sigma /= np.linalg.norm(sigma, axis=1, keepdims=True)
    kw = dict(N=8, L=4.0, masses=(1.0, 2.0), omega=0.74, alpha=1.4, N_rho=2, sigma=sigma,
              w_sigma=np.full(5, 4 * np.pi / 5))
    f = _inputs(8, 4.0, (1.0, 2.0), 2, seed=93)
    assert check(gpu_collision(f, precision=precision, **kw), oracle_collision(f, **kw), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vss_negated_design(precision):
    """The icosahedron with every direction negated: the stored direction of each antipodal
    pair (the lower index) is now the one a halved self pair does not use, so the self pairs
    and the reused (j,i) outputs take the other side of the conjugate symmetry
    F(k, rho, -sigma) = conj F(k, rho, sigma)."""
    sigma, w = quadrature.spherical_design(12)
    kw = dict(N=8, L=4.0, masses=(1.0, 1.7, 3.0), omega=0.74, alpha=1.4, N_rho=2, sigma=-sigma,
              w_sigma=w)
    f = _inputs(8, 4.0, (1.0, 1.7, 3.0), 2, seed=95)
    assert check(gpu_collision(f, precision=precision, **kw), oracle_collision(f, **kw), precision)


@pytest.mark.parametrize("antipodal", [True, False])
def test_vss_table_holds_one_slot_per_antipodal_pair(antipodal):
    """F(k, rho, -sigma) = conj F(k, rho, sigma): the FP32 gain table holds one complex slot
    per (pair, rho) and antipodal pair of directions, and one per direction without an
    antipode: M/2 for the icosahedron, M/2 + 1 once one direction is moved off its antipode."""
    N, s, M, NR = 8, 2, 12, 3
    sigma, w = quadrature.spherical_design(M)
    if not antipodal:
        sigma = sigma.copy()
        sigma[0] = np.array([0.6, 0.0, 0.8])   # breaks the antipode of one direction
    plan = dgfs.Plan(N, 4.0, [1.0, 2.0], 0.74, alpha=1.4, M=M, N_rho=NR, precision="fp32",
                     sigma=sigma, w_sigma=w)
    tables, _ = plan.bytes(0)
    plan.close()
    slots = M // 2 if antipodal else M // 2 + 1
    gain = s * s * NR * slots * N ** 3 * 8
    loss = s * s * N ** 3 * 4
    assert gain + loss <= tables < gain + loss + (1 << 20)
