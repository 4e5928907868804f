"""Seeded synthetic inputs shared by the tests and bench.py.

Holds no solver arithmetic: meshes (element widths), GLL sample positions for
evaluating right-hand sides, random skeleton vectors and right-hand sides.
The paper's test cases are analytic or pseudo-random (Sec. 5.2), so nothing
here stands in for a dataset.

Workloads (names used by bench.py and the tests):
  poisson_4x4x4_p4        lambda = 0, n = 4, p = 4, f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)
  helmholtz_8x8x8_p{4,8,16,32}
                          lambda = 1, n = 8, f = (1 + 3 pi^2) sss + N(0, sigma = 1e-2), seed 1808035952
  helmholtz_16x16x16_p16  lambda in {0, 100}, f ~ U(-1, 1), seed 1808035953
  poisson_6x6x6_p48_stretched
                          lambda = 0, per-axis widths exp(U(0, ln 8)) normalised to 1 (seed 1808035954),
                          manufactured f
  poisson_2x2x2_p48_stretched
                          the same degree, width law, seed and f on 2 x 2 x 2 elements: the bounded
                          sample of the 6^3 workload that the oracle is timed on
  expansion_widths(n, alpha)
                          per-axis widths in geometric progression on (0, 2 pi), the stretched
                          meshes of the paper's iteration-count table (Sec. 5.4)
  paper_sec52_8x8x8_p{16,32}
                          paper_solution on 8^3 uniform elements of (0, 2 pi)^3, k = 5, lambda = 0,
                          Dirichlet data u_ex at all faces (the problem of the runtime tests, Sec. 5.2)
  paper_solution(h, p, k, lam)
                          the manufactured solution of the paper's runtime tests (Sec. 5.2) on
                          (0, 2 pi)^3 with inhomogeneous Dirichlet data: (u_ex, f = lam u_ex - Laplace u_ex)
                          at the GLL nodes, k = 5 in the paper
  batch64                 64 solves, n ~ U{2..12}, p ~ U{4..24}, lambda = 10^U(-2, 3), f ~ U(-1, 1),
                          seed 1808035955
"""
import math

import numpy as np
from numpy.polynomial import legendre as _leg

SEED_CFG2 = 1808035952
SEED_CFG3 = 1808035953
SEED_CFG4 = 1808035954
SEED_CFG5 = 1808035955


def gll_sample_points(p):
    """Reference GLL positions on [-1, 1] at which a nodal right-hand side is sampled."""
    if p == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(p + 1)
    c[p] = 1.0
    x = np.sort(np.real(_leg.legroots(_leg.legder(c))))
    d1, d2 = _leg.legder(c), _leg.legder(c, 2)
    for _ in range(4):
        x = x - _leg.legval(x, d1) / _leg.legval(x, d2)
    return np.concatenate([[-1.0], x, [1.0]])


def node_coords(h, p):
    """Global GLL node coordinates per axis for per-axis widths h[d] (origin 0)."""
    xi = gll_sample_points(p)
    out = []
    for hd in h:
        hd = np.asarray(hd, float)
        X = np.concatenate([[0.0], np.cumsum(hd)])
        x = np.zeros(len(hd) * p + 1)
        for a in range(len(hd)):
            x[a * p:(a + 1) * p + 1] = X[a] + 0.5 * hd[a] * (xi + 1.0)
        out.append(x)
    return out


def uniform_widths(n, length=1.0):
    return [np.full(n, length / n) for _ in range(3)]


def stretched_widths(n, seed=SEED_CFG4, ratio=8.0):
    """Per-axis widths with ratios drawn log-uniform in [1, ratio], each axis normalised to length 1."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(3):
        w = np.exp(rng.uniform(0.0, math.log(ratio), size=n))
        out.append(w / w.sum())
    return out


def expansion_widths(n, alpha, length=2 * math.pi):
    """Per-axis widths growing by the constant factor alpha from one end of each axis to the other
    (the paper's stretched test meshes, Sec. 5.4: largest over smallest width alpha^(n-1))."""
    w = alpha ** np.arange(n, dtype=float)
    return [length * w / w.sum() for _ in range(3)]


def sinsinsin(h, p):
    x = node_coords(h, p)
    X3, X2, X1 = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    return np.sin(np.pi * X1) * np.sin(np.pi * X2) * np.sin(np.pi * X3)


def manufactured_rhs(h, p, lam):
    """f = (lam + 3 pi^2) sin(pi x) sin(pi y) sin(pi z) at the GLL nodes (unit cube)."""
    return (lam + 3 * np.pi**2) * sinsinsin(h, p)


# u_ex of Sec. 5.2 as a product of five plane waves trig(k (a . x + b)): (is_cos, a, b)
_PAPER_FACTORS = ((True, (1.0, -3.0, 2.0), 0.0), (False, (1.0, 0.0, 0.0), 1.0), (False, (0.0, -1.0, 0.0), 1.0),
                  (False, (2.0, 1.0, 0.0), 0.0), (False, (3.0, -2.0, 2.0), 0.0))


def paper_solution_at(X1, X2, X3, k, lam):
    """(u_ex, f) of Sec. 5.2 at points (X1, X2, X3).  With u = prod_i phi_i, phi_i = trig(theta_i),
    theta_i = k (a_i . x + b_i):  Laplace u = -k^2 sum_i |a_i|^2 u + 2 k^2 sum_{i<j} (a_i . a_j) phi_i' phi_j'
    prod_{l != i, j} phi_l, phi' the derivative of trig."""
    X = (X1, X2, X3)
    val, der, aa = [], [], []
    for is_cos, a, b in _PAPER_FACTORS:
        th = k * (a[0] * X[0] + a[1] * X[1] + a[2] * X[2] + b)
        val.append(np.cos(th) if is_cos else np.sin(th))
        der.append(-np.sin(th) if is_cos else np.cos(th))
        aa.append(np.asarray(a))
    u = np.prod(val, axis=0)
    lap = -k * k * sum(float(a @ a) for a in aa) * u
    nf = len(val)
    for i in range(nf):
        for j in range(i + 1, nf):
            rest = np.prod([val[l] for l in range(nf) if l not in (i, j)], axis=0)
            lap = lap + 2.0 * k * k * float(aa[i] @ aa[j]) * der[i] * der[j] * rest
    return u, lam * u - lap


def paper_solution(h, p, k=5.0, lam=0.0):
    """(u_ex, f) of Sec. 5.2 at the GLL nodes of the mesh with widths h (arrays [g3, g2, g1])."""
    x = node_coords(h, p)
    X3, X2, X1 = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    return paper_solution_at(X1, X2, X3, k, lam)


def random_nodal(h, p, seed, kind="normal"):
    rng = np.random.default_rng(seed)
    shape = tuple(len(hd) * p + 1 for hd in reversed(h))
    if kind == "uniform":
        return rng.uniform(-1.0, 1.0, size=shape)
    return rng.standard_normal(shape)


def config(name, p=None, lam=None):
    """(widths, p, lam, f_nodal, p0) of a named workload."""
    if name == "poisson_4x4x4_p4":
        h = uniform_widths(4)
        return h, 4, 0.0, manufactured_rhs(h, 4, 0.0), 1
    if name.startswith("helmholtz_8x8x8"):
        p = int(name.rsplit("_p", 1)[1]) if p is None else p
        h = uniform_widths(8)
        rng = np.random.default_rng(SEED_CFG2 + p)
        f = manufactured_rhs(h, p, 1.0)
        f = f + rng.normal(0.0, 1e-2, size=f.shape)
        return h, p, 1.0, f, 2
    if name == "helmholtz_16x16x16_p16":
        lam = 0.0 if lam is None else lam
        h = uniform_widths(16)
        return h, 16, lam, random_nodal(h, 16, SEED_CFG3, "uniform"), 2
    if name in ("poisson_6x6x6_p48_stretched", "poisson_2x2x2_p48_stretched"):
        h = stretched_widths(int(name.split("_")[1][0]))
        return h, 48, 0.0, manufactured_rhs(h, 48, 0.0), 2
    raise KeyError(name)


def batch64(seed=SEED_CFG5, count=64):
    """The 64 independent solves of the batched workload: list of (widths, p, lam, f)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(2, 13))
        p = int(rng.integers(4, 25))
        lam = float(10.0 ** rng.uniform(-2.0, 3.0))
        h = uniform_widths(n)
        f = random_nodal(h, p, seed + 1 + i, "uniform")
        out.append((h, p, lam, f))
    return out
