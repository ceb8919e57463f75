"""The plan builder's host logic on the CPU (no GPU): task lists, entry weights, sigma_x
groups, y-pass sharing flags and the slot codes of the VSS gain table, read back through a
small probe linked against libdgfs.so.  The GPU parity tests exercise the same lists end to
end; here each rule is checked on its own."""

import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import quadrature
from paper_1903_03056_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers")
    lib = build.build()
    exe = str(tmp_path_factory.mktemp("probe") / "plan_probe")
    libdir = os.path.dirname(lib)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", build.CSRC,
                    "-I", CUDA_INC, os.path.join(ROOT, "tests", "plan_probe.cpp"), "-o", exe,
                    "-L", libdir, "-ldgfs", "-Wl,-rpath," + libdir], check=True)

    def run(N=8, L=4.0, masses=(1.0, 2.0), omega=0.7, alpha=1.0, M=12, N_rho=3, precision=1,
            flags=0, sigma=None, w_sigma=None, R=0.0):
        s = len(masses)
        om = np.broadcast_to(np.asarray(omega, dtype=float), (s, s)).reshape(-1)
        al = np.broadcast_to(np.asarray(alpha, dtype=float), (s, s)).reshape(-1)
        if sigma is not None:
            M = len(sigma)
            if w_sigma is None:
                w_sigma = np.full(M, 4 * np.pi / M)
        words = [N, repr(float(L)), s, precision, flags, N_rho, M, int(sigma is not None), repr(float(R))]
        words += [repr(float(x)) for x in masses] + [repr(float(x)) for x in om]
        words += [repr(float(x)) for x in al]
        if sigma is not None:
            words += [repr(float(x)) for x in np.asarray(sigma, dtype=float).reshape(-1)]
            words += [repr(float(x)) for x in w_sigma]
        out = subprocess.run([exe], input=" ".join(str(w) for w in words), capture_output=True,
                             text=True, check=True).stdout
        return json.loads(out)

    return run


def _sigma(plan, m):
    return np.array(plan["sigma"][3 * m:3 * m + 3])


def test_antipodal_rule_gives_unordered_tasks_with_halved_self_pairs(probe):
    p = probe(masses=(1.0, 2.0, 3.0), M=12)
    assert p["rc"] == 0 and p["antipodal"] == 1
    pairs = [(t["i"], t["j"]) for t in p["tasks"]]
    assert pairs == [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
    for t in p["tasks"]:
        assert t["out0"] == 3 * t["i"] + t["j"]
        n = len(t["entries"])
        if t["i"] == t["j"]:
            # p(sigma) = p(-sigma): half the directions, doubled weights (VHS)
            assert t["out1"] == -1 and n == 6
            assert all(abs(e["w"] - 2 * 4 * np.pi / 12) < 1e-14 for e in t["entries"])
        else:
            # the (j,i) output is served by the same products
            assert t["out1"] == 3 * t["j"] + t["i"] and n == 12
        assert abs(sum(e["w"] for e in t["entries"]) - 4 * np.pi) < 1e-12


def test_non_antipodal_rule_gives_every_ordered_pair(probe):
    rng = np.random.default_rng(1)
    sig = rng.normal(size=(5, 3))
    sig /= np.linalg.norm(sig, axis=1, keepdims=True)
    p = probe(sigma=sig)
    assert p["antipodal"] == 0
    assert [(t["i"], t["j"]) for t in p["tasks"]] == [(0, 0), (0, 1), (1, 0), (1, 1)]
    assert all(t["out1"] == -1 and len(t["entries"]) == 5 for t in p["tasks"])


def test_per_pair_radius_keeps_halving_but_not_reuse(probe):
    p = probe(flags=8)
    assert [(t["i"], t["j"]) for t in p["tasks"]] == [(0, 0), (0, 1), (1, 0), (1, 1)]
    for t in p["tasks"]:
        assert t["out1"] == -1
        assert len(t["entries"]) == (6 if t["i"] == t["j"] else 12)
    R = np.array(p["pair_R"]).reshape(2, 2)
    assert abs(p["R"] - R.min()) < 1e-12 and R.max() > R.min()


@pytest.mark.parametrize("alpha", [1.0, 1.4])
def test_groups_share_sigma_x_and_ysh_marks_repeated_sigma_y(probe, alpha):
    p = probe(alpha=alpha, M=12)
    for t in p["tasks"]:
        ents = t["entries"]
        covered = []
        for first, count in t["groups"]:
            covered += list(range(first, first + count))
            sx = {round(_sigma(p, ents[e]["m"])[0], 12) for e in range(first, first + count)}
            assert len(sx) == 1                       # one sigma_x per group
            if alpha != 1.0:
                assert count == 1                     # VSS: one forward transform per entry
        assert covered == list(range(len(ents)))
        xs = [_sigma(p, e["m"])[0] for e in ents]
        assert xs == sorted(xs)                       # entries ordered by sigma_x
        for k, e in enumerate(ents):
            same = k > 0 and np.allclose(_sigma(p, ents[k - 1]["m"])[:2], _sigma(p, e["m"])[:2])
            assert e["ysh"] == (1 if same and alpha == 1.0 else 0)


def test_vss_slot_codes(probe):
    """One table slot per antipodal pair (the lower index owns it); the antipode reads it
    conjugated (bit 0); a halved self pair reads without conjugation and marks the sum with
    the antipode's code; a cross pair's reused output reads the antipode's slot."""
    p = probe(alpha=1.4, M=12)
    M = 12
    sig = np.array(p["sigma"]).reshape(M, 3)
    anti = [int(np.argmin(np.linalg.norm(sig + sig[m], axis=1))) for m in range(M)]
    assert p["n_fslot"] == 6
    for m in range(M):
        code = p["fslot"][m]
        if anti[m] > m:
            assert code % 2 == 0
        else:
            assert code == p["fslot"][anti[m]] + 1
    assert sorted({c // 2 for c in p["fslot"]}) == list(range(6))
    for t in p["tasks"]:
        for e in t["entries"]:
            m = e["m"]
            if t["i"] == t["j"]:
                assert e["code0"] == p["fslot"][m] & ~1
            else:
                assert e["code0"] == p["fslot"][m]
            assert e["code1"] == p["fslot"][anti[m]]


def test_vss_slot_codes_with_duplicates_and_broken_antipodes(probe):
    """Directions whose negation does not own a slot get a slot of their own; a repeated
    direction reads the same slot as its first copy's antipode would."""
    sig, _ = quadrature.spherical_design(6)
    sig = sig.copy()
    sig[0] = [0.6, 0.0, 0.8]                          # +x moved: -x loses its antipode
    p = probe(alpha=1.4, sigma=sig)
    assert p["antipodal"] == 0 and p["n_fslot"] == 4  # (+-y), (+-z) share; moved +x, -x alone
    dup = np.concatenate([quadrature.spherical_design(6)[0], [[0.0, 0.0, -1.0]]])
    q = probe(alpha=1.4, sigma=dup)
    codes = q["fslot"]
    # the repeated -z reads the +z slot conjugated, like the first -z
    iz = [k for k in range(6) if np.allclose(dup[k], [0, 0, 1])][0]
    assert codes[6] == codes[iz] + 1 and q["n_fslot"] == 3


def test_invalid_descriptions_fail_in_the_builder(probe):
    assert probe(N=10)["rc"] == -2
    assert probe(omega=0.3)["rc"] == -1
    assert probe(flags=8, R=3.0)["rc"] == -1


@pytest.mark.parametrize("R", [0.0, 12.0])
def test_vss_rule_size_converges_at_the_plans_largest_argument(probe, R):
    """The plan sizes the t rule of the VSS gain weight from the table's largest argument
    a = pi rho c_j |k| / L.  On the N = 48 three-species workload (a ~ 65) it keeps 64 points;
    a user radius of 12 pushes a past 140 and the rule grows.  At that argument and at every
    angle, the plan's rule agrees with the oracle's converged integral to 1e-13 of the bound."""
    from oracle import kernel
    p = probe(N=48, L=8.0, masses=(1.0, 1.5, 2.6), omega=0.74, alpha=1.4, M=32, N_rho=24, R=R)
    assert p["rc"] == 0 and p["vss"] == 1
    a = p["vss_a_max"]
    if R == 0.0:
        assert 60.0 < a < 65.3 and p["n_t"] == 64
    else:
        assert a > 140.0 and p["n_t"] > 64
    cos_t = np.linspace(-1.0, 1.0, 21)
    plan_rule = kernel.phi_integral(a, cos_t, 1.4, p["n_t"])
    converged = kernel.phi_integral(a, cos_t, 1.4, kernel.jacobi_rule_size(a, 1.4))
    assert np.max(np.abs(plan_rule - converged)) < 1e-13 * 2 ** 1.4 / 1.4


def test_bf16x3_plans_accept_vhs_on_n_up_to_24_only(probe):
    """The tensor-core precision (code 2) builds VHS plans on N = 8, 16, 24; other N return
    DGFS_ERR_UNSUPPORTED_N (-2) and alpha != 1 DGFS_ERR_UNSUPPORTED (-7), before any device work."""
    assert probe(N=24, masses=(1.0, 4.0), omega=0.5, precision=2)["rc"] == 0
    assert probe(N=8, precision=2)["rc"] == 0
    assert probe(N=32, precision=2)["rc"] == -2
    assert probe(N=12, precision=2)["rc"] == -2
    assert probe(N=16, alpha=1.4, precision=2)["rc"] == -7
    assert probe(N=16, precision=3)["rc"] == -1
