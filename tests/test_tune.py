"""The launch-shape tuner's host logic: its mirror of the kernel geometry and the shapes the
library is built with (CPU)."""

import os
import re

from paper_1903_03056_gb300 import tune


def _committed_shapes():
    text = open(tune.SHAPES_H).read()
    out = []
    for m in re.finditer(r"^DGFS_SHAPE(3?)\((float|double), (\d+), (\d+), (\d+)(?:, (\d+))?\)$", text, re.M):
        T, N, C, GP = m.group(2), int(m.group(3)), int(m.group(4)), int(m.group(5))
        MB = int(m.group(6)) if m.group(6) else 1
        out.append((T, N, C, GP, MB))
    return out


def test_every_supported_size_has_a_shape_per_precision():
    shapes = _committed_shapes()
    for T in ("float", "double"):
        assert sorted(N for t, N, *_ in shapes if t == T) == [4, 6, 8, 12, 16, 24, 32, 48]


def test_committed_shapes_are_valid():
    for T, N, C, GP, MB in _committed_shapes():
        assert tune.valid(N, C, GP, MB, 8 if T == "float" else 16), (T, N, C, GP, MB)


def test_geometry_mirrors_the_kernel_rules():
    # FP32 keeps P in registers up to N = 48, FP64 up to N = 16
    assert tune.geometry(48, 4, 4, 1, 8)["preg"] and not tune.geometry(24, 2, 6, 1, 16)["preg"]
    # y-pass sharing only at N <= 16, and then a third plane buffer per group
    g16 = tune.geometry(16, 1, 8, 3, 8)
    assert g16["ysh"] and g16["nbuf"] == 3 and g16["res"] == 3
    g32 = tune.geometry(32, 2, 4, 1, 8)
    assert not g32["ysh"] and g32["nbuf"] == 2 and g32["res"] == 2
    assert g32["smem"] == 4 * 2 * 32 * 33 * 8   # 66 KB of plane buffers per CTA
    # P in shared memory: three buffers per group
    assert tune.geometry(32, 4, 4, 1, 16)["nbuf"] == 3
    # tensor-memory accumulators: one plane per group in 8-CTA clusters at 3 CTAs per SM
    # (3 x 128 of the 512 columns) keep only the transpose buffer; four planes per group
    # (2-CTA clusters) would need 320 columns a CTA, so that shape keeps P in registers
    g = tune.geometry(32, 8, 4, 3, 8)
    assert g["tm"] and g["nbuf"] == 1 and g["smem"] == 4 * 32 * 33 * 8
    assert not tune.geometry(32, 2, 4, 1, 8)["tm"] and tune.geometry(32, 4, 4, 2, 8)["tm"]
    assert not tune.geometry(32, 8, 4, 3, 16)["tm"] and not tune.geometry(48, 4, 4, 1, 8)["tm"]


def test_shape_line_round_trip():
    line = tune._shape_line("float", 32, 2, 4, 1)
    assert line == "DGFS_SHAPE3(float, 32, 2, 4, 1)"
    text = open(tune.SHAPES_H).read()
    assert tune._patch(text, "float", 32, line).count(line) == 1
    assert os.path.exists(tune.SHAPES_JSON)


def _committed_radix():
    text = open(tune.RADIX_H).read()
    return [(m.group(1), int(m.group(2)), int(m.group(3)))
            for m in re.finditer(r"^DGFS_RADIX\((float|double), (\d+), (\d+)\)$", text, re.M)]


def test_every_supported_size_has_a_valid_radix_schedule_per_precision():
    rows = _committed_radix()
    for T in ("float", "double"):
        assert sorted(N for t, N, _ in rows if t == T) == [4, 6, 8, 12, 16, 24, 32, 48]
    for T, N, code in rows:
        assert tune.radix_code_valid(N, code), (T, N, code)


def test_radix_candidates_are_orders_of_valid_schedules():
    for N, codes in tune.RADIX_CANDIDATES.items():
        assert len(set(codes)) == len(codes)
        for code in codes:
            assert tune.radix_code_valid(N, code), (N, code)
        assert not tune.radix_code_valid(N, codes[0] * 10 + 2)
