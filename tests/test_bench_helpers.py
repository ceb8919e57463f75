"""The bench's algorithmic work counts (every reported TFLOP/s and roofline fraction rests on
them), checked against an explicit enumeration of the method's transforms."""

import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_1903_03056_gb300 import synth  # noqa: E402


def _enumerate_transforms(w):
    """Count 3D transforms by walking the evaluation of one node (Sec. 4): forward transform of
    each species; per unordered pair, per radial node and per design direction the two shifted
    inverse transforms, except that with an antipodal design the (j,i) products equal the (i,j)
    ones and a self pair needs half the directions; the forward transforms of the products
    (VHS: one per radial node and unordered pair after the sigma sum; VSS: one per product);
    the two inverse transforms (gain and loss) of every ordered pair."""
    n = 0
    n += w.s                                      # f_hat of every species
    for i in range(w.s):
        for j in range(i, w.s):
            dirs = w.M // 2 if i == j else w.M    # self pair: p(sigma) = p(-sigma)
            n += 2 * w.N_rho * dirs               # a and b per (rho, sigma)
            if w.alpha == 1.0:
                n += w.N_rho                      # sigma-summed product, one per rho
            else:
                n += w.N_rho * dirs               # every product on its own
    n += 2 * w.s * w.s                            # gain and loss inverse transforms
    return n


@pytest.mark.parametrize("key", sorted(synth.WORKLOADS))
def test_transform_count_matches_enumeration(key):
    w = synth.WORKLOADS[key]
    assert bench.transforms_per_node(w) == _enumerate_transforms(w)


def test_bench_workload_flops():
    w = synth.WORKLOADS["dg_batch_n32"]
    assert bench.transforms_per_node(w) == 826
    n3 = 32 ** 3
    assert bench.flops_per_transform(32) == 5 * n3 * math.log2(n3)
    assert abs(bench.transforms_per_node(w) * bench.flops_per_transform(32) - 2.0299776e9) < 1.0


def test_reference_arm_line(capsys, monkeypatch):
    """`bench.py --impl reference`: the oracle on the host cores, W untimed and K timed steps,
    one JSON line with the reference keys (on the small single-node workload here)."""
    import argparse
    import json
    monkeypatch.delenv("RANK", raising=False)
    args = argparse.Namespace(gpus=1, steps=2, warmup=1)
    line = bench.reference_arm(args, key="single_node_n16")
    printed = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert printed == line
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["unit"] == "evals/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1 and line["dtype"] == "f64"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"] == {"value": line["value"], "unit": "evals/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import argparse
    monkeypatch.setenv("RANK", "1")
    assert bench.reference_arm(argparse.Namespace(gpus=2, steps=1, warmup=0)) is None
    assert capsys.readouterr().out == ""


def test_bf16x3_tensor_work_counts_the_kernels_transforms():
    """The tensor-core kernel recomputes f_hat per task (one per species of the task), does two
    shifted transforms per entry and radial node (self pairs: half the directions), one forward
    transform of the product sum per radial node, and a loss and a gain transform per output
    pair; every transform is 3 passes of ceil(N^2/128) tiles x 6 split products of
    2 x 128 x 2N x 2N flop."""
    w = synth.WORKLOADS["hs_n24"]
    n = 0
    for i in range(w.s):
        for j in range(i, w.s):
            nspec = 1 if i == j else 2
            entries = w.M // 2 if i == j else w.M
            outputs = 1 if i == j else 2
            n += nspec + 2 * entries * w.N_rho + w.N_rho + 2 * outputs
    transforms, flops = bench.bf16x3_tensor_flops_per_node(w)
    assert transforms == n == 624
    assert flops == n * 3 * math.ceil(w.N * w.N / 128) * 6 * 2 * 128 * (2 * w.N) ** 2
