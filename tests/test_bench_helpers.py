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
