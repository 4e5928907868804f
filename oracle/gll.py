"""1D Gauss-Lobatto-Legendre (GLL) basis in FP64 -- oracle, test infrastructure only.

Sec. 2.1: the standard-element mass matrix is the GLL-quadrature (hence diagonal)
mass matrix and the standard-element stiffness matrix is the exact Galerkin
stiffness of the Lagrange polynomials through the GLL nodes, both of size
(p+1) x (p+1) on the reference interval [-1, 1].

Everything here is computed from first principles:
  * nodes: -1, the roots of P_p' (Legendre), +1; polished by Newton's method;
  * weights: w_i = 2 / (p (p+1) P_p(x_i)^2);
  * Lagrange derivatives and interpolation: barycentric formulas;
  * stiffness: L = D^T diag(w) D, exact because (l_i' l_j') has degree 2p-2
    and GLL quadrature with p+1 nodes is exact to degree 2p-1.
"""
import functools

import numpy as np
from numpy.polynomial import legendre as npleg


@functools.lru_cache(maxsize=None)
def gll(p):
    """GLL nodes x[0..p] (ascending) and weights w[0..p] for degree p >= 1."""
    if p < 1:
        raise ValueError("degree must be >= 1")
    if p == 1:
        return np.array([-1.0, 1.0]), np.array([1.0, 1.0])
    cP = np.zeros(p + 1)
    cP[p] = 1.0
    dP = npleg.legder(cP)
    d2P = npleg.legder(dP)
    x = np.sort(np.real(npleg.legroots(dP)))
    for _ in range(4):  # Newton polish of the roots of P_p'
        x = x - npleg.legval(x, dP) / npleg.legval(x, d2P)
    x = np.concatenate([[-1.0], x, [1.0]])
    w = 2.0 / (p * (p + 1) * npleg.legval(x, cP) ** 2)
    x.setflags(write=False)
    w.setflags(write=False)
    return x, w


def bary_weights(x):
    """Barycentric weights b_j = 1 / prod_{k != j} (x_j - x_k)."""
    x = np.asarray(x, float)
    diff = x[:, None] - x[None, :]
    np.fill_diagonal(diff, 1.0)
    return 1.0 / np.prod(diff, axis=1)


def diff_matrix(x):
    """D[i, j] = l_j'(x_i) for the Lagrange basis through the nodes x."""
    x = np.asarray(x, float)
    b = bary_weights(x)
    n = len(x)
    D = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i != j:
                D[i, j] = (b[j] / b[i]) / (x[i] - x[j])
        D[i, i] = -np.sum(D[i, :])
    return D


def interp_matrix(x_from, x_to):
    """J[i, j] = l_j(x_to[i]) for the Lagrange basis through the nodes x_from."""
    x_from = np.asarray(x_from, float)
    x_to = np.asarray(x_to, float)
    b = bary_weights(x_from)
    J = np.zeros((len(x_to), len(x_from)))
    for i, t in enumerate(x_to):
        d = t - x_from
        hit = np.flatnonzero(d == 0.0)
        if hit.size:
            J[i, hit[0]] = 1.0
            continue
        c = b / d
        J[i, :] = c / np.sum(c)
    return J


@functools.lru_cache(maxsize=None)
def standard_matrices(p):
    """Standard-element mass M_S = diag(w) and stiffness L_S = D^T diag(w) D (Sec. 2.1)."""
    x, w = gll(p)
    D = diff_matrix(x)
    M = np.diag(w)
    L = D.T @ M @ D
    L = 0.5 * (L + L.T)
    M.setflags(write=False)
    L.setflags(write=False)
    return M, L


def weight_poly(t):
    """Smooth 1D Schwarz weight of degree p_W = 7 (Sec. 3.2, smoother weights).

    The paper asks for a polynomial of degree 7 that is one at the own vertex
    (t = 0), zero at the other vertex (t = 1), with higher derivatives zero at
    both vertices.  Derivatives 1..3 vanishing at t = 0 and t = 1 plus the two
    end values are 8 conditions, which fix w(t) = 1 - 35t^4 + 84t^5 - 70t^6 + 20t^7
    uniquely (w'(t) = -140 t^3 (1-t)^3).
    """
    t = np.asarray(t, float)
    return 1.0 - 35.0 * t**4 + 84.0 * t**5 - 70.0 * t**6 + 20.0 * t**7
