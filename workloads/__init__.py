"""Seeded synthetic workloads for the parametrized diffusion problems.

This module only *describes* problems and *draws* random numbers.  It holds
none of the method's arithmetic (no operator, no solver, no projection), so
both the FP64 oracle and the CUDA library can take their inputs from it
without sharing any computation.

Problem family (the paper's eq. 1 with the affine form of eq. 12):
    -div(kappa(x; mu) grad u) = f(x; mu) on the unit square / cube,
    u = 0 on the boundary, kappa = mu_p on block p of a box partition,
    f = sum_r phi_r(mu) f_r.
The grid, block partition and load terms of each workload are plain data
here; the discretisation itself is written independently in `oracle/` and in
the CUDA kernels.

The paper's two test cases (Section 5, Table 1) are finite-difference analogues
of the same family with coefficient FIELDS instead of blocks:
    kappa(x; mu) = sum_q theta_q F_q(x)   (F_q given at the nodes),
    u = g(x; mu) on the boundary, lifted into load terms.
For them this module evaluates the fields, the source and the boundary data at
the nodes (input data, like the Gaussian bumps' parameters) and maps the
physical parameters of the paper's domain to the affine coefficients theta_q,
phi_r that both the oracle and the library take as the parameter vector.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014, "Fast
splittable pseudorandom number generators"): state += 0x9E3779B97F4A7C15,
then two xor-shift-multiply rounds.  A double in [0, 1) is (z >> 11) * 2^-53.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` consecutive SplitMix64 outputs of the stream that starts at `seed`."""
    out = np.empty(count, dtype=np.uint64)
    s = seed & _MASK
    for i in range(count):
        s = (s + _GOLDEN) & _MASK
        z = s
        z = ((z ^ (z >> 30)) * _M1) & _MASK
        z = ((z ^ (z >> 27)) * _M2) & _MASK
        out[i] = z ^ (z >> 31)
    return out


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2^-53."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass(frozen=True)
class Load:
    """One load term f_r of f(mu) = sum_r phi_r(mu) f_r.

    kind  : "const" (f_r = 1 at every node), "gauss"
            (f_r(x) = exp(-|x - center|^2 / (2 sigma^2)) at node coordinates),
            "array" (f_r = the node values of the source `recipe`) or
            "boundary" (the lift of the Dirichlet data `recipe` through the
            coefficient field `field`: the boundary faces' terms F_field(i) g(j) / h^2
            moved to the right-hand side).
    param : -1 means phi_r = 1; otherwise phi_r = mu[param].
    """
    kind: str
    param: int = -1
    center: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    sigma: float = 0.0
    recipe: str = ""
    field: int = 0


@dataclasses.dataclass(frozen=True)
class Problem:
    """Grid, block partition and load terms of one parametrized diffusion problem.

    dims        : interior nodes per direction, (mx, my) or (mx, my, mz); x fastest.
    blocks      : blocks per direction; P = prod(blocks) diffusion parameters.
    loads       : load terms; mu has P + n_load_params entries.
    coefficient : "blocks" (kappa = mu_p on block p) or the name of a field recipe
                  (kappa = sum_q mu_q F_q(x), P = number of fields; blocks are all 1).
    """
    dims: Tuple[int, ...]
    blocks: Tuple[int, ...]
    loads: Tuple[Load, ...]
    coefficient: str = "blocks"

    @property
    def dim(self) -> int:
        return len(self.dims)

    @property
    def n_dof(self) -> int:
        return int(np.prod(self.dims))

    @property
    def P(self) -> int:
        if self.coefficient != "blocks":
            return len(FIELD_RECIPES[self.coefficient])
        return int(np.prod(self.blocks))

    def field_values(self) -> np.ndarray | None:
        """[P][N_dof] node values of the coefficient fields (None for block coefficients)."""
        if self.coefficient == "blocks":
            return None
        return _field_values(self.dims, self.coefficient)

    def load_values(self, r: int) -> np.ndarray | None:
        """Values of an "array" load at the nodes [N_dof], or of a "boundary" load's Dirichlet
        data on the grid extended by the boundary layer [(mz+2)][(my+2)][(mx+2)] (x fastest);
        None for the other kinds."""
        ld = self.loads[r]
        if ld.kind == "array":
            return _source_values(self.dims, ld.recipe)
        if ld.kind == "boundary":
            return _boundary_values(self.dims, ld.recipe)
        return None

    @property
    def n_mu(self) -> int:
        extra = [ld.param for ld in self.loads if ld.param >= 0]
        return max([self.P - 1] + extra) + 1


@dataclasses.dataclass(frozen=True)
class Workload:
    """A named workload: problem, basis size and the seeded parameter sets."""
    name: str
    problem: Problem
    n_basis: int
    mu_range: Tuple[float, float]          # log-uniform range of the P block values
    load_range: Tuple[float, float]        # uniform range of the load parameters
    n_train: int
    n_test: int
    batch: int
    train_seed: int = 1
    test_seed: int = 2
    bump_seed: int = 3
    case: str = ""                         # "case1" / "case2": parameters drawn in the paper's domain

    def draw_physical(self, seed: int, count: int) -> np.ndarray:
        """count x d physical parameters of a paper case, uniform in its domain (Section 5:
        [0, 1] for Case 1, [0, 2] x [0, 1] for Case 2)."""
        dom = CASE_DOMAINS[self.case]
        u = uniform01(seed, count * len(dom)).reshape(count, len(dom))
        lo = np.array([a for a, _ in dom])
        hi = np.array([b for _, b in dom])
        return lo + u * (hi - lo)

    def draw_mu(self, seed: int, count: int) -> np.ndarray:
        """count x n_mu parameter vectors from stream `seed`.

        Each vector draws n_mu uniforms in order; the first P become
        exp(ln a + u (ln b - ln a)) (log-uniform block values), the rest
        lo + u (hi - lo) (load parameters).  For a paper case the vectors are the
        affine coefficients case_theta(physical parameters).
        """
        if self.case:
            return np.stack([case_theta(self.case, m) for m in self.draw_physical(seed, count)])
        P, n_mu = self.problem.P, self.problem.n_mu
        u = uniform01(seed, count * n_mu).reshape(count, n_mu)
        a, b = self.mu_range
        mu = np.empty_like(u)
        mu[:, :P] = np.exp(math.log(a) + u[:, :P] * (math.log(b) - math.log(a)))
        lo, hi = self.load_range
        mu[:, P:] = lo + u[:, P:] * (hi - lo)
        return mu

    def train_mu(self) -> np.ndarray:
        return self.draw_mu(self.train_seed, self.n_train)

    def test_mu(self, count: int | None = None) -> np.ndarray:
        return self.draw_mu(self.test_seed, self.n_test if count is None else count)


def bump_centers(seed: int, count: int, dim: int, lo: float = 0.2, hi: float = 0.8) -> np.ndarray:
    """count x dim Gaussian-bump centres, uniform in [lo, hi]^dim."""
    u = uniform01(seed, count * dim).reshape(count, dim)
    return lo + u * (hi - lo)


def _const_load() -> Tuple[Load, ...]:
    return (Load("const"),)


def _bump_loads(seed: int, dim: int, P: int, sigma: float = 0.05) -> Tuple[Load, ...]:
    c = bump_centers(seed, 2, dim)
    pad = lambda v: tuple(float(t) for t in v) + (0.0,) * (3 - dim)
    return (Load("const"),
            Load("gauss", param=P + 0, center=pad(c[0]), sigma=sigma),
            Load("gauss", param=P + 1, center=pad(c[1]), sigma=sigma))


def rbi_2d_64() -> Workload:
    """2D, 64x64 interior grid, 2x2 blocks, f = 1, n = 20, 200 train / 50 test."""
    prob = Problem(dims=(64, 64), blocks=(2, 2), loads=_const_load())
    return Workload("rbi_2d_64x64_P4_n20", prob, n_basis=20, mu_range=(0.1, 10.0),
                    load_range=(0.0, 1.0), n_train=200, n_test=50, batch=50)


def rbcg_2d_512() -> Workload:
    """2D, 512x512 interior grid, 3x3 blocks, f = 1 + mu_9 f_1 + mu_10 f_2, n = 40."""
    P = 9
    prob = Problem(dims=(512, 512), blocks=(3, 3), loads=_bump_loads(3, 2, P))
    return Workload("rbcg_2d_512x512_P9_n40", prob, n_basis=40, mu_range=(0.1, 10.0),
                    load_range=(0.0, 1.0), n_train=1000, n_test=1000, batch=1000)


def batched_3d_128() -> Workload:
    """3D, 128^3 interior grid, 2x2x2 blocks, f = 1, n = 60, 256 queries per launch."""
    prob = Problem(dims=(128, 128, 128), blocks=(2, 2, 2), loads=_const_load())
    return Workload("rbcg_3d_128cube_P8_n60", prob, n_basis=60, mu_range=(0.1, 10.0),
                    load_range=(0.0, 1.0), n_train=512, n_test=256, batch=256)


def ragged_3d(m: int) -> Workload:
    """3D m^3 member of the ragged batch (m in 64, 96, 128), 2x2x2 blocks, n = 60."""
    prob = Problem(dims=(m, m, m), blocks=(2, 2, 2), loads=_const_load())
    return Workload(f"rbcg_3d_{m}cube_P8_n60", prob, n_basis=60, mu_range=(0.1, 10.0),
                    load_range=(0.0, 1.0), n_train=512, n_test=256, batch=256)


def large_3d_256() -> Workload:
    """3D, 256^3 interior grid, 3x3x3 blocks, mu in [0.01, 100], f = 1, n = 100."""
    prob = Problem(dims=(256, 256, 256), blocks=(3, 3, 3), loads=_const_load())
    return Workload("rbcg_3d_256cube_P27_n100", prob, n_basis=100, mu_range=(0.01, 100.0),
                    load_range=(0.0, 1.0), n_train=512, n_test=64, batch=64)


def small(dims: Sequence[int], blocks: Sequence[int], n_basis: int, n_train: int = 40,
          bumps: bool = False, mu_range=(0.1, 10.0), name: str | None = None) -> Workload:
    """A small problem of the same family, for tests that must finish in seconds."""
    dims, blocks = tuple(dims), tuple(blocks)
    P = int(np.prod(blocks))
    loads = _bump_loads(3, len(dims), P) if bumps else _const_load()
    prob = Problem(dims=dims, blocks=blocks, loads=loads)
    nm = name or ("small_" + "x".join(map(str, dims)) + "_P%d_n%d" % (P, n_basis))
    return Workload(nm, prob, n_basis=n_basis, mu_range=mu_range, load_range=(0.0, 1.0),
                    n_train=n_train, n_test=16, batch=16)


# ---------------------------------------------------------------------------
# The paper's test cases (Section 5, Table 1) on finite-difference grids.
#
#   Case 1: kappa = 1 + mu r^2, r^2 = sum_d (x_d - 1/2)^2, g = 0, mu in [0, 1]
#           -> A(mu) = A_1 + mu A_2 (fields F_0 = 1, F_1 = r^2), theta = (1, mu).
#   Case 2: kappa = 1 + mu_1 sin^2(20 pi s(x)), s = 4 (x - 1/2)^2 + sum_{d>0} (x_d - 1/2)^2,
#           g = (1 - mu_2) cos(10 pi s(x)) + mu_2 cos(10 pi sum_d x_d), mu in [0, 2] x [0, 1]
#           -> A(mu) = A_1 + mu_1 A_2, and the lift of g through kappa(mu) gives four load
#           terms besides the source, with phi = (1 - mu_2), mu_1 (1 - mu_2), mu_2, mu_1 mu_2.
#   Both: source f = d pi^2 prod_d sin(pi x_d) (the paper's 3 pi^2 sin sin sin in 3D; the
#   sign is that of the SPD form -div(kappa grad u) = f).

CASE_DOMAINS = {"case1": ((0.0, 1.0),), "case2": ((0.0, 2.0), (0.0, 1.0))}


def _coords(dims, extended: bool):
    """Node coordinates per direction (x first): interior nodes (i + 1) h, or the grid extended by
    the boundary layer, e h for e = 0 .. m + 1; each array broadcastable to the grid shape."""
    out = []
    nd = len(dims)
    for d, m in enumerate(dims):
        shape = [1] * nd
        shape[nd - 1 - d] = m + 2 if extended else m
        e = np.arange(m + 2) if extended else np.arange(m) + 1.0
        out.append((e / (m + 1.0)).reshape(shape))
    return out


def _s(c):
    """4 (x - 1/2)^2 + sum over the other directions of (x_d - 1/2)^2."""
    return 4.0 * (c[0] - 0.5) ** 2 + sum((cd - 0.5) ** 2 for cd in c[1:])


def _product(factors):
    out = 1.0
    for f in factors:
        out = out * f
    return out


def _r2(c):
    return sum((cd - 0.5) ** 2 for cd in c)


FIELD_RECIPES = {
    "case1": (lambda c: np.ones_like(_r2(c)), _r2),
    "case2": (lambda c: np.ones_like(_r2(c)), lambda c: np.sin(20.0 * math.pi * _s(c)) ** 2),
}
SOURCE_RECIPES = {
    "sine": lambda c: len(c) * math.pi ** 2 * _product(np.sin(math.pi * cd) for cd in c),
}
BOUNDARY_RECIPES = {
    "case2_a": lambda c: np.cos(10.0 * math.pi * _s(c)),
    "case2_b": lambda c: np.cos(10.0 * math.pi * sum(c)),
}


def _grid(dims, v, extended: bool):
    shape = tuple(reversed([m + 2 if extended else m for m in dims]))
    return np.broadcast_to(v, shape).reshape(-1).astype(np.float64)


def _field_values(dims, name):
    c = _coords(dims, False)
    return np.stack([_grid(dims, f(c), False) for f in FIELD_RECIPES[name]])


def _source_values(dims, name):
    return _grid(dims, SOURCE_RECIPES[name](_coords(dims, False)), False)


def _boundary_values(dims, name):
    return _grid(dims, BOUNDARY_RECIPES[name](_coords(dims, True)), True)


def case_theta(case: str, m) -> np.ndarray:
    """Affine coefficients (theta_q of A, then the load weights) of a case's physical parameters."""
    if case == "case1":
        return np.array([1.0, float(m[0])])
    if case == "case2":
        m1, m2 = float(m[0]), float(m[1])
        return np.array([1.0, m1, 1.0 - m2, m1 * (1.0 - m2), m2, m1 * m2])
    raise ValueError(case)


def case_problem(case: str, dims: Sequence[int]) -> Problem:
    dims = tuple(dims)
    blocks = (1,) * len(dims)
    src = Load("array", recipe="sine")
    if case == "case1":
        return Problem(dims=dims, blocks=blocks, loads=(src,), coefficient="case1")
    if case == "case2":
        lift = [Load("boundary", param=2 + 2 * j + q, recipe=g, field=q)
                for j, g in enumerate(("case2_a", "case2_b")) for q in (0, 1)]
        return Problem(dims=dims, blocks=blocks, loads=(src, *lift), coefficient="case2")
    raise ValueError(case)


def paper_case(case: str, m: int = 64, dim: int = 3, n_basis: int = 20, n_train: int = 200,
               n_test: int = 100) -> Workload:
    """The paper's Case 1 / Case 2 on an m^dim interior grid (100 test parameters, as in the
    paper's convergence study)."""
    prob = case_problem(case, (m,) * dim)
    name = f"{case}_{dim}d_{m}_n{n_basis}"
    return Workload(name, prob, n_basis=n_basis, mu_range=(1.0, 1.0), load_range=(0.0, 1.0),
                    n_train=n_train, n_test=n_test, batch=n_test, case=case)


WORKLOADS = {
    "rbi_2d_64": rbi_2d_64,
    "rbcg_2d_512": rbcg_2d_512,
    "batched_3d_128": batched_3d_128,
    "batched_3d_64": lambda: ragged_3d(64),
    "large_3d_256": large_3d_256,
    "case1_3d_64": lambda: paper_case("case1", 64),
    "case2_3d_64": lambda: paper_case("case2", 64),
    "case1_3d_128": lambda: paper_case("case1", 128, n_test=256),
}


def load_arrays(problem: Problem):
    """Flatten the load descriptors to arrays (kind code, param, centre, sigma).

    kind code: 0 = const, 1 = gauss, 2 = array, 3 = boundary.  This is a format conversion for the
    C interface, not arithmetic of the method.
    """
    kinds = np.array([{"const": 0, "gauss": 1, "array": 2, "boundary": 3}[ld.kind] for ld in problem.loads],
                     dtype=np.int32)
    params = np.array([ld.param for ld in problem.loads], dtype=np.int32)
    centers = np.array([ld.center for ld in problem.loads], dtype=np.float64).reshape(-1, 3)
    sigmas = np.array([ld.sigma for ld in problem.loads], dtype=np.float64)
    return kinds, params, centers, sigmas


# ---------------------------------------------------------------------------
# Learned warm start: seeded draws only (initial weights and the parameter
# vectors of the training pairs).  The network's arithmetic lives in oracle/ and
# in the CUDA library.

MLP_INIT_SEED = 4
MLP_TRAIN_SEED = 5
TUNE_SEED = 6       # the autotuner's sample: neither the greedy's training set nor the test queries


def tune_mu(w: "Workload", count: int) -> np.ndarray:
    """Parameter vectors the autotuner times (the workload's distribution, own stream).  Training
    parameters would bias it: the greedy's snapshots are exact in the basis, so a start from the RB
    approximation converges at once for them."""
    return w.draw_mu(TUNE_SEED, count)


def mlp_layer_sizes(n_in: int, n_out: int, hidden: int = 128) -> Tuple[int, ...]:
    """Widths of the warm-start network: n_in -> hidden -> hidden -> n_out."""
    return (n_in, hidden, hidden, n_out)


def mlp_init(sizes: Sequence[int], seed: int = MLP_INIT_SEED):
    """Initial weights and biases, layer by layer: W_l [out][in] uniform in
    [-a, a] with a = sqrt(6 / (in + out)) (Glorot-uniform), biases zero.
    Returns a list of (W_l, b_l) float64 arrays."""
    out = []
    for l in range(len(sizes) - 1):
        fi, fo = sizes[l], sizes[l + 1]
        a = math.sqrt(6.0 / (fi + fo))
        u = uniform01(seed * 1000 + l, fi * fo).reshape(fo, fi)
        out.append(((2.0 * u - 1.0) * a, np.zeros(fo)))
    return out


def mlp_train_mu(w: "Workload", count: int, seed: int = MLP_TRAIN_SEED) -> np.ndarray:
    """Parameter vectors of the warm-start training pairs (the workload's distribution)."""
    return w.draw_mu(seed, count)
