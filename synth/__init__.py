"""Seeded synthetic instances of the mixed dense-sparse (MDS) problem class.

This module only draws inputs.  It holds none of the interior-point method's
arithmetic and is the one piece of code that both the CPU oracle and the GPU
path consume (they share nothing else).

Problem class (Section 2, Eqs. (obj)-(bounds)), variables ordered x = [x_s; x_d]:

    min  0.5 x_d^T Q x_d + sum_i 0.25 x_s,i^4 + c^T x
    s.t. x_s,i - x_s,i+m_E + a_i^T x_d = b_i           i = 0..m_E-1  (g, equalities)
         ||x_d[S_j]||^2 <= r_j                          j = 0..m_I-1  (h, inequalities)
         -1 <= x_s <= 1,   x_d free

with n_s = 2 m_E, Q = G^T G / n_d + 0.1 I, G ~ N(0,1), c ~ U(-1,1),
a_i ~ N(0, sigma_a^2), b ~ U(-0.5, 0.5).  With m_I = 1 the single inequality
covers all of x_d with r = 4; otherwise a random permutation of x_d is split
into m_I chunks of floor(n_d/m_I) indices, each with r = 1.

The sparse Jacobian block J_sg is returned as COO triplets (row i has +1 at
column i and -1 at column i+m_E), the inequality block J_sh is empty, and the
Hessian of the sparse block is diagonal (assumptions A1/A2 of Section 2).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["Instance", "CONFIGS", "make_instance", "make_config", "random_iterate", "FAMILY",
           "family_rhs", "draw_family_params", "mlp_init"]


@dataclasses.dataclass
class Instance:
    n_d: int
    n_s: int
    m_E: int
    m_I: int
    Q: np.ndarray          # (n_d, n_d) symmetric positive definite
    c: np.ndarray          # (n_s + n_d,)
    A: np.ndarray          # (m_E, n_d) row-major, dense Jacobian block J_{x_d} g
    b: np.ndarray          # (m_E,)   equality right-hand side g_E
    Jsg_rows: np.ndarray   # (nnz,) int32
    Jsg_cols: np.ndarray   # (nnz,) int32 (column index into x_s)
    Jsg_vals: np.ndarray   # (nnz,) float64
    h_set: np.ndarray      # (n_d,) int32: index j of the inequality that x_d[k] enters, -1 if none
    hu: np.ndarray         # (m_I,) upper bounds r_j of h_j
    hl: np.ndarray         # (m_I,) lower bounds (-inf)
    xl: np.ndarray         # (n,) lower bounds (-inf = none)
    xu: np.ndarray         # (n,) upper bounds (+inf = none)
    x0: np.ndarray         # (n,) starting point
    name: str = ""
    # sparse block J_sh of the inequalities (COO, empty in the benchmark family)
    Jsh_rows: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    Jsh_cols: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0, np.int32))
    Jsh_vals: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))

    @property
    def n(self) -> int:
        return self.n_s + self.n_d

    @property
    def m(self) -> int:
        return self.m_E + self.m_I


# (n_d, m_E, m_I, sigma_a) of the benchmark family; n_s = 2 m_E.
CONFIGS = {
    0: dict(n_d=32, m_E=1000, m_I=1, sigma_a=0.1),        # plain FP64, reduced matrix 1033^2
    1: dict(n_d=2000, m_E=100000, m_I=50, sigma_a=0.01),  # plain FP64, OPF-like scale
    2: dict(n_d=4000, m_E=200000, m_I=50, sigma_a=0.01),  # mixed-precision scale
    4: dict(n_d=512, m_E=25600, m_I=50, sigma_a=0.01),    # parametric family (warm start)
}

# Parametric family for the learned warm start: the instance of CONFIGS[4]
# (seed 4) with b = b0 (1 + 0.2 p[block(i)]), p in R^64 ~ U(-1, 1), and
# block(i) = i // 400 (64 blocks of 400 equality rows).
FAMILY = dict(config=4, n_p=64, amplitude=0.2)


def make_instance(n_d: int, m_E: int, m_I: int, sigma_a: float, seed: int,
                  name: str = "", q_shift: float = 0.1, jsh_per_row: int = 0) -> Instance:
    """Draw one instance.  Everything is a pure function of the arguments.

    q_shift is the multiple of I added to G^T G / n_d (0.1 in the benchmark
    family); a negative value makes Q indefinite, a nonconvex variant whose
    x_d is still confined by the inequalities when every x_d is covered.

    jsh_per_row > 0 adds a sparse linear part to every inequality,
    h_j(x) = ||x_d[S_j]||^2 + sum_{a in T_j} e_ja x_s,a, with T_j that many
    distinct x_s indices and e_ja ~ U(-0.5, 0.5): a nonzero J_sh (its Hessian
    stays zero, so assumption A2 holds).  Those draws come from a stream of
    their own (seeded by (seed, 1)), so the rest of the instance is the same
    as without them.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_s = 2 * m_E
    n = n_s + n_d
    G = rng.standard_normal((n_d, n_d))
    Q = G.T @ G / n_d + q_shift * np.eye(n_d)
    Q = 0.5 * (Q + Q.T)
    c = rng.uniform(-1.0, 1.0, size=n)
    A = rng.standard_normal((m_E, n_d))
    A *= sigma_a
    b = rng.uniform(-0.5, 0.5, size=m_E)
    rows = np.concatenate([np.arange(m_E), np.arange(m_E)]).astype(np.int32)
    cols = np.concatenate([np.arange(m_E), np.arange(m_E) + m_E]).astype(np.int32)
    vals = np.concatenate([np.ones(m_E), -np.ones(m_E)])
    h_set = -np.ones(n_d, dtype=np.int32)
    if m_I == 1:
        h_set[:] = 0
        hu = np.array([4.0])
    elif m_I > 1:
        perm = rng.permutation(n_d)
        chunk = n_d // m_I
        for j in range(m_I):
            h_set[perm[j * chunk:(j + 1) * chunk]] = j
        hu = np.ones(m_I)
    else:
        hu = np.zeros(0)
    hl = np.full(m_I, -np.inf)
    xl = np.concatenate([-np.ones(n_s), np.full(n_d, -np.inf)])
    xu = np.concatenate([np.ones(n_s), np.full(n_d, np.inf)])
    x0 = np.zeros(n)
    inst = Instance(n_d=n_d, n_s=n_s, m_E=m_E, m_I=m_I, Q=Q, c=c, A=np.ascontiguousarray(A),
                    b=b, Jsg_rows=rows, Jsg_cols=cols, Jsg_vals=vals, h_set=h_set, hu=hu,
                    hl=hl, xl=xl, xu=xu, x0=x0, name=name)
    if jsh_per_row > 0 and m_I > 0 and n_s > 0:
        rh = np.random.Generator(np.random.PCG64([seed, 1]))
        k = min(jsh_per_row, n_s)
        inst.Jsh_rows = np.repeat(np.arange(m_I), k).astype(np.int32)
        inst.Jsh_cols = np.concatenate([rh.choice(n_s, size=k, replace=False) for _ in range(m_I)]).astype(np.int32)
        inst.Jsh_vals = rh.uniform(-0.5, 0.5, size=m_I * k)
    return inst


def make_config(k: int, seed: int | None = None) -> Instance:
    """Benchmark family member k (seed defaults to k)."""
    p = CONFIGS[k]
    return make_instance(p["n_d"], p["m_E"], p["m_I"], p["sigma_a"],
                         seed=k if seed is None else seed, name=f"mds{k}")


def random_iterate(inst: Instance, seed: int, spread: float = 1.0) -> dict:
    """A strictly interior primal-dual point (for direction-parity checks).

    Bounded x_s lie in (-1, 1); bound multipliers are positive; d lies strictly
    inside its bounds.  `spread` widens the range of slacks/multipliers, which
    makes the Newton system worse conditioned.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n, m_I = inst.n, inst.m_I
    x = np.zeros(n)
    x[:inst.n_s] = rng.uniform(-0.9, 0.9, size=inst.n_s)
    x[inst.n_s:] = rng.uniform(-0.3, 0.3, size=inst.n_d)
    has_l = np.isfinite(inst.xl)
    has_u = np.isfinite(inst.xu)
    zl = np.where(has_l, np.exp(rng.uniform(-spread, spread, size=n)), 0.0)
    zu = np.where(has_u, np.exp(rng.uniform(-spread, spread, size=n)), 0.0)
    d = inst.hu - np.exp(rng.uniform(-spread, 0.0, size=m_I))
    vl = np.zeros(m_I)
    vu = np.exp(rng.uniform(-spread, spread, size=m_I))
    yg = rng.uniform(-1.0, 1.0, size=inst.m_E)
    yh = rng.uniform(0.0, 1.0, size=m_I)
    return dict(x=x, d=d, yg=yg, yh=yh, zl=zl, zu=zu, vl=vl, vu=vu)


def family_rhs(inst: Instance, p: np.ndarray, amplitude: float = 0.2) -> np.ndarray:
    """Equality right-hand side of family member p: b0 (1 + amplitude p[block(i)]).

    The m_E rows are cut into len(p) consecutive blocks of m_E // len(p) rows
    (the last block takes the remainder)."""
    p = np.asarray(p, dtype=np.float64)
    n_p = p.shape[0]
    size = max(1, inst.m_E // n_p)
    block = np.minimum(np.arange(inst.m_E) // size, n_p - 1)
    return inst.b * (1.0 + amplitude * p[block])


def draw_family_params(count: int, n_p: int, seed: int) -> np.ndarray:
    """count x n_p parameter vectors, i.i.d. U(-1, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=(count, n_p))


def mlp_init(n_in: int, n_hidden: int, n_out: int, seed: int, out_scale: float = 0.1) -> dict:
    """Initial weights of the warm-start network: uniform(-r, r) with
    r = sqrt(6 / fan_in) for the two hidden layers (He), r = out_scale
    sqrt(3 / fan_in) for the output layer; zero biases.  FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def u(rows, cols, r):
        return rng.uniform(-r, r, size=(rows, cols)).astype(np.float32)

    return dict(W1=u(n_hidden, n_in, np.sqrt(6.0 / n_in)), b1=np.zeros(n_hidden, np.float32),
                W2=u(n_hidden, n_hidden, np.sqrt(6.0 / n_hidden)), b2=np.zeros(n_hidden, np.float32),
                W3=u(n_out, n_hidden, out_scale * np.sqrt(3.0 / n_hidden)), b3=np.zeros(n_out, np.float32))
