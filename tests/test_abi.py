"""The C-ABI library builds, loads and exports every declared symbol; arguments are checked
before any device work.  Runs without a GPU."""

import ctypes
import os
import re

import pytest

from paper_1903_03056_gb300 import build, dgfs

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dgfs.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dgfs.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(dgfs_\w+)\(", text, flags=re.M)))


def test_header_declares_the_binding_names():
    assert set(declared_functions()) == set(dgfs.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def _desc(**kw):
    base = dict(N=16, L=6.0, masses=[1.0, 2.0], omega=0.5, M=6, N_rho=8, precision="fp64")
    base.update(kw)
    N, L, masses, omega = base.pop("N"), base.pop("L"), base.pop("masses"), base.pop("omega")
    return dgfs.make_desc(N, L, masses, omega, **base)


@pytest.mark.parametrize("kw,code", [
    (dict(N=10), dgfs.DGFS_ERR_UNSUPPORTED_N),
    (dict(N=64), dgfs.DGFS_ERR_UNSUPPORTED_N),
    (dict(L=0.0), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(omega=0.3), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(alpha=2.5), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(M=7), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(N_rho=0), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(masses=[1.0, -2.0]), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(sigma=[[0.0, 0.0, 2.0]]), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(flags=16), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(flags=8, R=4.0), dgfs.DGFS_ERR_INVALID_ARG),   # per-pair truncation computes its own R
    (dict(kappa=[1.0, float("nan"), 1.0, 1.0], flags=2), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(b_override=[1.0, float("inf"), 1.0, 1.0]), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(R=float("inf")), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(M=6, sigma=[[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
          w_sigma=[1.0, float("nan"), 1.0, 1.0, 1.0, 1.0]), dgfs.DGFS_ERR_INVALID_ARG),
])
def test_invalid_plans_rejected_before_device_work(lib, kw, code):
    desc, keep = _desc(**kw)
    got, handle = dgfs.dgfs_create_plan(desc)
    assert got == code and handle is None


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.dgfs_create_plan(None, ctypes.byref(h)) == dgfs.DGFS_ERR_INVALID_ARG
    assert dgfs.dgfs_eval_collision(None, None, None, 1, None) == dgfs.DGFS_ERR_INVALID_ARG
    assert dgfs.dgfs_eval_collision_host(None, None, None, 1, None) == dgfs.DGFS_ERR_INVALID_ARG
    assert dgfs.dgfs_destroy_plan(None) == dgfs.DGFS_ERR_INVALID_ARG
    assert dgfs.dgfs_plan_radius(None)[0] == dgfs.DGFS_ERR_INVALID_ARG
    assert dgfs.dgfs_plan_check(None)[0] == dgfs.DGFS_ERR_INVALID_ARG


def test_strerror_names_every_code(lib):
    codes = [v for k, v in vars(dgfs).items() if k.startswith("DGFS_ERR_")] + [0]
    names = {dgfs.dgfs_strerror(c) for c in codes}
    assert len(names) == len(codes) and "unknown error" not in names
