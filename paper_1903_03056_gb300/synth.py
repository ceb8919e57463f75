"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the collision method: it only samples distribution
functions on the velocity grid.  Both the CUDA path and the CPU oracle are fed from it.

Grid: cell-centred nodes v_n = -L + (n + 1/2) 2L/N on each axis; arrays are laid out
[node][species][x][y][z] with z fastest.

The base shape is the nondimensional Maxwellian of Sec. 3,
    M(v; n, u, T, m) = n (m / (pi T))^(3/2) exp(-m |v - u|^2 / T),
with, per node, species and component, n ~ U[0.5, 1.5], u ~ U[-0.5, 0.5]^3,
T ~ U[0.7, 1.3].  Every node draws from its own PCG64 stream seeded with seed0 + node.
"""

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One collision workload: grid, species, kernel, quadrature sizes and input recipe."""
    name: str
    batch: int
    N: int
    L: float
    masses: tuple
    omega: float
    alpha: float
    M: int
    N_rho: int
    recipe: str            # "bimaxwellian" | "skewed"
    noise: float = 0.0     # multiplicative uniform noise amplitude
    seed0: int = 0
    extra: dict = field(default_factory=dict, compare=False, hash=False)

    @property
    def s(self):
        return len(self.masses)


# The paper's parameter ranges (Table 1 and the flow cases of Sec. 6) shape these.
SINGLE_NODE_N16 = Workload("single-node N=16 2-species VHS FP64", 1, 16, 6.0, (1.0, 2.0),
                           0.5, 1.0, 6, 8, "bimaxwellian", 0.0, 1000)
DG_BATCH_N32 = Workload("4096 DG nodes N=32 2-species VHS", 4096, 32, 7.0, (1.0, 2.1),
                        0.81, 1.0, 12, 16, "bimaxwellian", 0.05, 2000)
VSS_N48 = Workload("1024 DG nodes N=48 3-species VSS", 1024, 48, 8.0, (1.0, 1.5, 2.6),
                   0.74, 1.4, 32, 24, "skewed", 0.0, 3000)
HS_N24 = Workload("16384 DG nodes N=24 2-species HS", 16384, 24, 6.0, (1.0, 4.0),
                  0.5, 1.0, 12, 12, "bimaxwellian", 0.0, 4000)

# grids of the serving mix at fixed parameters (tuning and per-size measurements)
VHS_N16 = Workload("8192 DG nodes N=16 2-species VHS", 8192, 16, 6.0, (1.0, 2.0),
                   0.75, 1.0, 12, 8, "bimaxwellian", 0.05, 5000)
VHS_N48 = Workload("512 DG nodes N=48 3-species VHS", 512, 48, 8.0, (1.0, 1.5, 2.6),
                   0.75, 1.0, 12, 24, "bimaxwellian", 0.05, 6000)

WORKLOADS = {"single_node_n16": SINGLE_NODE_N16, "dg_batch_n32": DG_BATCH_N32,
             "vss_n48": VSS_N48, "hs_n24": HS_N24, "vhs_n16": VHS_N16, "vhs_n48": VHS_N48}


def grid(N, L):
    return -L + (2.0 * L / N) * (np.arange(N) + 0.5)


def maxwellian(N, L, n, u, T, m):
    v = grid(N, L)
    ex = np.exp(-m * (v - u[0]) ** 2 / T)
    ey = np.exp(-m * (v - u[1]) ** 2 / T)
    ez = np.exp(-m * (v - u[2]) ** 2 / T)
    return n * (m / (np.pi * T)) ** 1.5 * ex[:, None, None] * ey[None, :, None] * ez[None, None, :]


def _draw_state(rng):
    n = rng.uniform(0.5, 1.5)
    u = rng.uniform(-0.5, 0.5, size=3)
    T = rng.uniform(0.7, 1.3)
    return n, u, T


def node_distribution(w: Workload, node: int, N=None):
    """f[s, N, N, N] (float64) of one node of workload ``w``."""
    N = w.N if N is None else N
    rng = np.random.Generator(np.random.PCG64(w.seed0 + node))
    f = np.zeros((w.s, N, N, N))
    v = grid(N, w.L)
    for i, m in enumerate(w.masses):
        if w.recipe == "bimaxwellian":
            for _ in range(2):
                n, u, T = _draw_state(rng)
                f[i] += maxwellian(N, w.L, n, u, T, m)
        elif w.recipe == "skewed":
            # shifted Maxwellian times (1 + a (xi.e)(|xi|^2 - 5/2)), xi = sqrt(m/T)(v - u):
            # a Grad-type heat-flux term that leaves n, u and T unchanged
            n, u, T = _draw_state(rng)
            e = rng.normal(size=3)
            e /= np.linalg.norm(e)
            s = np.sqrt(m / T)
            xi = [s * (v - u[d]) for d in range(3)]
            X, Y, Z = np.meshgrid(*xi, indexing="ij")
            f[i] = maxwellian(N, w.L, n, u, T, m) * (
                1.0 + 0.05 * (X * e[0] + Y * e[1] + Z * e[2]) * (X * X + Y * Y + Z * Z - 2.5))
        else:
            raise ValueError(w.recipe)
        if w.noise > 0.0:
            f[i] *= 1.0 + w.noise * rng.uniform(-1.0, 1.0, size=f[i].shape)
    return np.maximum(f, 0.0)


def batch_distribution(w: Workload, nodes=None, dtype=np.float64):
    """f[len(nodes), s, N, N, N] for the listed nodes (default: all of the workload's batch)."""
    nodes = range(w.batch) if nodes is None else nodes
    nodes = list(nodes)
    out = np.empty((len(nodes), w.s, w.N, w.N, w.N), dtype=dtype)
    for k, b in enumerate(nodes):
        out[k] = node_distribution(w, b)
    return out
