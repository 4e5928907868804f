"""O1: dense / explicit-matrix FP64 oracle on tiny meshes -- test infrastructure only.

Problem (Sec. 2.1, eq. helmholtz_equation): lambda u - Laplace u = f on a box
meshed by a tensor product of cuboidal elements with per-axis widths h_d[a],
homogeneous Dirichlet conditions on all six faces, GLL nodal basis of degree p.

Conventions (readings of the paper, each stated where it is used):
  * nodal arrays are indexed u[g3, g2, g1] (C order, x1 fastest); the
    Kronecker product A3 (x) A2 (x) A1 acts with its rightmost factor along x1,
    so d_1 = h1 h2 h3 / 8 * 4 / h1^2 multiplies the stiffness along x1 (eq.
    helmholtzop read with that ordering);
  * condensed vectors are indexed by the ascending flat nodal index of the
    non-Dirichlet skeleton nodes (element-boundary nodes, Sec. 2.2);
  * the star of a vertex is every non-Dirichlet skeleton node strictly inside
    its 2x2x2 element block (Sec. 2.3, Fig. star; nodes +-p are the block's own
    homogeneous Dirichlet boundary and are dropped, n_S = 2p - 1).

Nothing here is fast; everything is meant to be checked against the paper by eye.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .gll import gll, interp_matrix, standard_matrices, weight_poly


class Mesh:
    """Tensor-product mesh: per-axis element widths h[d] (length n_d), degree p, lambda.

    bc: boundary condition of the faces -x1, +x1, -x2, +x2, -x3, +x3, each "D"
    (homogeneous Dirichlet, the default), "N" (homogeneous Neumann, Sec. 3.3:
    the boundary nodes are unknowns and the ghost element beyond the face is
    decoupled) or "P" (periodic, both faces of an axis, at least two elements
    along it: the ghost element is the element at the other end, Sec. 3.3).
    On a periodic axis the last node plane of a nodal array is the image of the
    first one (global node g and g + n_d p are the same unknown).
    """

    def __init__(self, h, p, lam, bc=None):
        self.h = [np.asarray(hd, dtype=float).copy() for hd in h]
        if len(self.h) != 3:
            raise ValueError("need three width arrays")
        self.n = [len(hd) for hd in self.h]
        self.p = int(p)
        self.lam = float(lam)
        self.N = [nd * self.p + 1 for nd in self.n]
        # vertex coordinates along each axis, origin at 0
        self.X = [np.concatenate([[0.0], np.cumsum(hd)]) for hd in self.h]
        self.bc = tuple(bc) if bc is not None else ("D",) * 6
        if len(self.bc) != 6 or any(b not in ("D", "N", "P") for b in self.bc):
            raise ValueError("bc: six entries, each 'D', 'N' or 'P'")
        for d in range(3):
            if (self.bc[2 * d] == "P") != (self.bc[2 * d + 1] == "P") or (self.bc[2 * d] == "P" and self.n[d] < 2):
                raise ValueError("periodic: both faces of an axis, with at least two elements along it")

    def with_degree(self, p):
        return Mesh(self.h, p, self.lam, self.bc)

    def periodic(self, d):
        return self.bc[2 * d] == "P"

    def g_range(self, d):
        """Global node indices [lo, hi] along axis d that are unknowns (not Dirichlet, not a periodic image)."""
        lo = 1 if self.bc[2 * d] == "D" else 0
        hi = self.N[d] - 2 if self.bc[2 * d + 1] in ("D", "P") else self.N[d] - 1
        return lo, hi

    def wrap(self, g, d):
        """Global node index along axis d, periodic images mapped to their unknown."""
        return np.mod(g, self.n[d] * self.p) if self.periodic(d) else g

    @property
    def shape(self):
        """Shape of a nodal array (N3, N2, N1)."""
        return (self.N[2], self.N[1], self.N[0])

    def node_coords(self):
        """Physical coordinates x_d[g] of the global GLL nodes along each axis."""
        xi, _ = gll(self.p)
        out = []
        for d in range(3):
            x = np.zeros(self.N[d])
            for a in range(self.n[d]):
                x[a * self.p:(a + 1) * self.p + 1] = self.X[d][a] + 0.5 * self.h[d][a] * (xi + 1.0)
            out.append(x)
        return out

    def flat(self, g1, g2, g3):
        return (np.asarray(g3) * self.N[1] + np.asarray(g2)) * self.N[0] + np.asarray(g1)

    def dirichlet_mask(self):
        """Nodal mask of the nodes on a Dirichlet face (where boundary values are prescribed)."""
        G3, G2, G1 = np.meshgrid(np.arange(self.N[2]), np.arange(self.N[1]), np.arange(self.N[0]), indexing="ij")
        m = np.zeros(self.shape, bool)
        for d, g in enumerate((G1, G2, G3)):
            if self.bc[2 * d] == "D":
                m |= g == 0
            if self.bc[2 * d + 1] == "D":
                m |= g == self.N[d] - 1
        return m


def element_operator(p, h1, h2, h3, lam):
    """Dense element Helmholtz operator, eq. helmholtzop with coefficients d_e (Sec. 2.1)."""
    M, L = standard_matrices(p)
    d0, d1, d2, d3 = (h1 * h2 * h3 / 8.0) * np.array([lam, 4.0 / h1**2, 4.0 / h2**2, 4.0 / h3**2])
    k = np.kron
    return d0 * k(M, k(M, M)) + d1 * k(M, k(M, L)) + d2 * k(M, k(L, M)) + d3 * k(L, k(M, M))


def sync_images(mesh, u):
    """Copy the first node plane of every periodic axis onto its image (last) plane."""
    u = np.array(u, dtype=float, copy=True)
    for d in range(3):
        if mesh.periodic(d):
            ax = 2 - d  # nodal arrays are [g3, g2, g1]
            first = np.take(u, [0], axis=ax)
            idx = [slice(None)] * 3
            idx[ax] = slice(u.shape[ax] - 1, u.shape[ax])
            u[tuple(idx)] = first
    return u


def _element_global_index(mesh, a1, a2, a3):
    p = mesh.p
    i = np.arange(p + 1)
    i3, i2, i1 = np.meshgrid(i, i, i, indexing="ij")
    return mesh.flat(mesh.wrap(a1 * p + i1, 0), mesh.wrap(a2 * p + i2, 1), mesh.wrap(a3 * p + i3, 2)).ravel()


def assemble_H(mesh):
    """Global operator H = sum_e Q_e H_e Q_e^T (Sec. 2.1), all nodes, as CSR."""
    rows, cols, vals = [], [], []
    for a3 in range(mesh.n[2]):
        for a2 in range(mesh.n[1]):
            for a1 in range(mesh.n[0]):
                He = element_operator(mesh.p, mesh.h[0][a1], mesh.h[1][a2], mesh.h[2][a3], mesh.lam)
                g = _element_global_index(mesh, a1, a2, a3)
                rows.append(np.repeat(g, len(g)))
                cols.append(np.tile(g, len(g)))
                vals.append(He.ravel())
    Nt = int(np.prod(mesh.N))
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(Nt, Nt))
    return H.tocsr()


def assemble_mass_diag(mesh):
    """Diagonal of the assembled GLL mass matrix (element mass (h1h2h3/8) M(x)M(x)M)."""
    _, w = gll(mesh.p)
    out = np.zeros(int(np.prod(mesh.N)))
    w3 = np.kron(w, np.kron(w, w))
    for a3 in range(mesh.n[2]):
        for a2 in range(mesh.n[1]):
            for a1 in range(mesh.n[0]):
                g = _element_global_index(mesh, a1, a2, a3)
                out[g] += mesh.h[0][a1] * mesh.h[1][a2] * mesh.h[2][a3] / 8.0 * w3
    return out


def index_sets(mesh):
    """Flat index sets: free (non-Dirichlet), B (free skeleton), I (element interiors)."""
    p = mesh.p
    g = [np.arange(Nd) for Nd in mesh.N]
    G3, G2, G1 = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    Gs = (G1, G2, G3)
    on_bdry = np.zeros(mesh.shape, bool)
    skel = np.zeros(mesh.shape, bool)
    for d in range(3):
        lo, hi = mesh.g_range(d)
        on_bdry |= (Gs[d] < lo) | (Gs[d] > hi)
        skel |= (Gs[d] % p == 0)
    free = ~on_bdry
    B = np.flatnonzero((free & skel).ravel())
    I = np.flatnonzero((free & ~skel).ravel())
    return {"free": np.flatnonzero(free.ravel()), "B": B, "I": I,
            "skel_mask": (free & skel), "G": Gs}


class Condensed:
    """Statically condensed system of Sec. 2.2 with explicit matrices.

    Hhat = H_BB - H_BI H_II^{-1} H_IB,  Fhat = F_B - H_BI H_II^{-1} F_I,
    u_I  = H_II^{-1} (F_I - H_IB u_B).
    """

    def __init__(self, mesh, dense=True):
        self.mesh = mesh
        sets = index_sets(mesh)
        self.B, self.I, self.free = sets["B"], sets["I"], sets["free"]
        H = assemble_H(mesh)
        self.H = H
        self.Hbb = H[self.B][:, self.B]
        self.Hbi = H[self.B][:, self.I]
        self.Hib = H[self.I][:, self.B]
        self.Hii = H[self.I][:, self.I].tocsc()
        self.lu_ii = spla.splu(self.Hii) if len(self.I) else None
        self.Mdiag = assemble_mass_diag(mesh)
        self.Hhat = None
        if dense:
            self.Hhat = self._schur()

    def _solve_ii(self, X):
        if self.lu_ii is None:
            return np.zeros((0,) + np.shape(X)[1:])
        return self.lu_ii.solve(np.asarray(X))

    def _schur(self):
        Hbb = self.Hbb.toarray()
        if len(self.I) == 0:
            return Hbb
        X = self._solve_ii(self.Hib.toarray())
        S = Hbb - self.Hbi @ X
        return 0.5 * (S + S.T)

    def apply(self, uB):
        """Hhat uB without forming Hhat (same definition, applied by solves)."""
        y = self.Hbb @ uB
        if len(self.I):
            y = y - self.Hbi @ self._solve_ii(self.Hib @ uB)
        return y

    def load(self, f_nodal):
        """F = M f with the assembled GLL mass (nodal f given at every GLL node)."""
        return self.Mdiag * np.asarray(f_nodal, float).ravel()

    def condense_rhs(self, F):
        F = np.asarray(F, float).ravel()
        Fh = F[self.B].copy()
        if len(self.I):
            Fh -= self.Hbi @ self._solve_ii(F[self.I])
        return Fh

    def recover(self, F, uB):
        """Nodal solution: u_B from the condensed system, u_I = H_II^{-1}(F_I - H_IB u_B); 0 on the Dirichlet
        boundary, periodic images set."""
        F = np.asarray(F, float).ravel()
        u = np.zeros(int(np.prod(self.mesh.N)))
        u[self.B] = uB
        if len(self.I):
            u[self.I] = self._solve_ii(F[self.I] - self.Hib @ uB)
        return sync_images(self.mesh, u.reshape(self.mesh.shape))

    def lifted_load(self, f_nodal, g_nodal):
        """Inhomogeneous Dirichlet data by lifting (Sec. 5.2 test problem): u = u_0 + E g with E g equal to g on
        the Dirichlet-face nodes and zero elsewhere, so H u_0 = M f - H E g with homogeneous conditions."""
        Eg = np.where(self.mesh.dirichlet_mask(), np.asarray(g_nodal, float), 0.0).ravel()
        return self.load(f_nodal) - self.H @ Eg

    def full_solve_dirichlet(self, f_nodal, g_nodal):
        """Exact discrete solution of H u = M f with u = g on the Dirichlet faces: the free rows of the
        uncondensed system with the prescribed values moved to the right-hand side."""
        dm = self.mesh.dirichlet_mask()
        u = np.where(dm, np.asarray(g_nodal, float), 0.0)
        return self.full_solve(self.lifted_load(f_nodal, g_nodal)) + u

    def full_solve(self, F):
        """Exact discrete solution of the uncondensed system H u = F (free nodes), nodal array."""
        F = np.asarray(F, float).ravel()
        Hff = self.H[self.free][:, self.free].tocsc()
        u = np.zeros(int(np.prod(self.mesh.N)))
        u[self.free] = spla.spsolve(Hff, F[self.free])
        return sync_images(self.mesh, u.reshape(self.mesh.shape))


# --------------------------------------------------------------------------
# Stars (Sec. 2.3, 3.1-3.3)
# --------------------------------------------------------------------------

def star_vertices(mesh):
    """All (n1+1)(n2+1)(n3+1) vertices, boundary ones included (Sec. 3.3); on a periodic
    axis the last vertex plane is the first one."""
    nv = [mesh.n[d] + (0 if mesh.periodic(d) else 1) for d in range(3)]
    return [(c1, c2, c3) for c3 in range(nv[2]) for c2 in range(nv[1]) for c1 in range(nv[0])]


def star_positions(mesh, B, c):
    """Positions in the condensed vector of the star nodes of vertex c, and their offsets j."""
    p = mesh.p
    g1 = B % mesh.N[0]
    g2 = (B // mesh.N[0]) % mesh.N[1]
    g3 = B // (mesh.N[0] * mesh.N[1])
    j = np.stack([g1 - c[0] * p, g2 - c[1] * p, g3 - c[2] * p], axis=1)
    for d in range(3):  # periodic axes: offset to the nearest image of the vertex
        if mesh.periodic(d):
            Lp = mesh.n[d] * p
            j[:, d] = np.mod(j[:, d] + Lp // 2, Lp) - Lp // 2
    inside = np.all(np.abs(j) <= p - 1, axis=1)
    pos = np.flatnonzero(inside)
    return pos, j[pos]


def assembled_1d(mesh, d):
    """Assembled 1D mass and stiffness along axis d: sum_a (h/2) M_S and (2/h) L_S."""
    M, L = standard_matrices(mesh.p)
    p, Nd = mesh.p, mesh.N[d]
    Mg = np.zeros((Nd, Nd))
    Lg = np.zeros((Nd, Nd))
    for a in range(mesh.n[d]):
        g = mesh.wrap(np.arange(a * p, (a + 1) * p + 1), d)
        Mg[np.ix_(g, g)] += 0.5 * mesh.h[d][a] * M
        Lg[np.ix_(g, g)] += 2.0 / mesh.h[d][a] * L
    return Mg, Lg


def star_line_table(mesh, d, c):
    """1D block eigen-table of vertex line c along axis d (Sec. 3.2 and 3.3).

    Block nodes g = c p + j, j = -(p-1)..(p-1).  A node is active when it is an
    unknown of the domain (inside the mesh and not on a Dirichlet face);
    inactive nodes (ghost element, Dirichlet vertex) are decoupled by padding S
    with identity and Lambda with 1.
    Returns S (n_S x n_S) with S^T M S = I, S^T L S = Lambda on the active block,
    Lambda (n_S) and the active mask.
    """
    p = mesh.p
    m = p - 1
    nS = 2 * m + 1
    Mg, Lg = assembled_1d(mesh, d)
    g = mesh.wrap(c * p + np.arange(-m, m + 1), d)
    lo, hi = mesh.g_range(d)
    active = (g >= lo) & (g <= hi)
    S = np.eye(nS)
    lam = np.ones(nS)
    ia = np.flatnonzero(active)
    if ia.size:
        ga = g[ia]
        ev, V = sla.eigh(Lg[np.ix_(ga, ga)], Mg[np.ix_(ga, ga)])
        S[np.ix_(ia, ia)] = V
        lam[ia] = ev
    return S, lam, active


def alg1_star_inverse(tables, F1, F2, F3, lam):
    """Algorithm 1: apply the inverse condensed star operator to a star residual.

    tables : [(S_d, Lambda_d, active_d)] for d = 1, 2, 3
    F1[j2, j3], F2[j1, j3], F3[j1, j2] : residual on the three star planes
        (perpendicular to x1, x2, x3), each n_S x n_S; a node on two or three
        planes carries its value on each of them.
    Returns the solution on the three planes (same layout).

    Steps, in the order of Algorithm 1:
      1. divide by the multiplicity (number of planes a node lies on);
      2. map each plane into the 3D eigenspace, expanding along its normal with
         the vertex row of S (eq. fast_diagonalization restricted to the planes);
      3. divide by the 3D eigenvalues D = lambda + Lambda_1 + Lambda_2 + Lambda_3
         (the geometric factors d_e are inside the assembled 1D matrices);
      4. map back to each plane with the transposed factors.
    """
    (S1, L1, _), (S2, L2, _), (S3, L3, _) = tables
    nS = S1.shape[0]
    m = (nS - 1) // 2
    z = np.arange(nS) == m
    mult1 = 1.0 + z[:, None] + z[None, :]          # on F1 the other two offsets are (j2, j3)
    F1 = F1 / mult1
    F2 = F2 / mult1
    F3 = F3 / mult1
    s1, s2, s3 = S1[m, :], S2[m, :], S3[m, :]      # vertex rows (offset 0)
    A1 = S2.T @ F1 @ S3                            # A1[k2, k3]
    A2 = S1.T @ F2 @ S3                            # A2[k1, k3]
    A3 = S1.T @ F3 @ S2                            # A3[k1, k2]
    E = (s1[:, None, None] * A1[None, :, :]
         + s2[None, :, None] * A2[:, None, :]
         + s3[None, None, :] * A3[:, :, None])     # E[k1, k2, k3]
    D = lam + L1[:, None, None] + L2[None, :, None] + L3[None, None, :]
    V = E / D
    B1 = np.einsum("a,abc->bc", s1, V)
    B2 = np.einsum("b,abc->ac", s2, V)
    B3 = np.einsum("c,abc->ab", s3, V)
    return S2 @ B1 @ S3.T, S1 @ B2 @ S3.T, S1 @ B3 @ S2.T


def star_planes_from_values(j, vals, nS):
    """Place star node values (offsets j) on the three planes, each node on every plane it lies on."""
    m = (nS - 1) // 2
    F = [np.zeros((nS, nS)) for _ in range(3)]
    for (j1, j2, j3), v in zip(j, vals):
        if j1 == 0:
            F[0][j2 + m, j3 + m] = v
        if j2 == 0:
            F[1][j1 + m, j3 + m] = v
        if j3 == 0:
            F[2][j1 + m, j2 + m] = v
    return F


def star_values_from_planes(j, F):
    """Read star node values back from the planes; a node on several planes gets their mean."""
    nS = F[0].shape[0]
    m = (nS - 1) // 2
    out = np.zeros(len(j))
    for k, (j1, j2, j3) in enumerate(j):
        acc, cnt = 0.0, 0
        if j1 == 0:
            acc += F[0][j2 + m, j3 + m]
            cnt += 1
        if j2 == 0:
            acc += F[1][j1 + m, j3 + m]
            cnt += 1
        if j3 == 0:
            acc += F[2][j1 + m, j2 + m]
            cnt += 1
        out[k] = acc / cnt
    return out


def star_weights(mesh, B, c, pos):
    """Weights W_i at the star nodes of vertex c (Sec. 3.2, weights; Fig. weights).

    W = product over axes of w(t_d), t_d = distance from the vertex along axis d
    divided by the width of the element on that side of the vertex, w the
    degree-7 weight polynomial.  Computed from physical coordinates.
    """
    x = mesh.node_coords()
    g1 = B[pos] % mesh.N[0]
    g2 = (B[pos] // mesh.N[0]) % mesh.N[1]
    g3 = B[pos] // (mesh.N[0] * mesh.N[1])
    W = np.ones(len(pos))
    for d, g in enumerate((g1, g2, g3)):
        xv = mesh.X[d][c[d]]
        dist = x[d][g] - xv
        if mesh.periodic(d):
            # the image of the vertex on the side the node's index offset points to
            Lp = mesh.n[d] * mesh.p
            j = np.mod(g - c[d] * mesh.p + Lp // 2, Lp) - Lp // 2
            per = mesh.X[d][-1]
            dist = np.where((j > 0) & (dist < 0), dist + per, np.where((j < 0) & (dist > 0), dist - per, dist))
            side = np.mod(np.where(j >= 0, c[d], c[d] - 1), mesh.n[d])
        else:
            side = np.where(dist >= 0, c[d], c[d] - 1)
        side = np.clip(side, 0, mesh.n[d] - 1)
        t = np.abs(dist) / mesh.h[d][side]
        W *= weight_poly(t)
    return W


def smoother_dense(mesh, cond, r, use_alg1=False):
    """Algorithm 2: Delta u = sum_i R_i^T W_i Hhat_i^{-1} R_i r over all vertices.

    Hhat_i = R_i Hhat R_i^T (Sec. 2.3, eq. smoother_definition); its inverse is
    applied densely (the precomputed-inverse idea) or, with use_alg1, by
    Algorithm 1 on the explicit 1D tables.
    """
    du = np.zeros_like(r)
    p = mesh.p
    nS = 2 * p - 1
    for c in star_vertices(mesh):
        pos, j = star_positions(mesh, cond.B, c)
        if pos.size == 0:
            continue
        if use_alg1:
            tabs = [star_line_table(mesh, d, c[d]) for d in range(3)]
            F = star_planes_from_values(j, r[pos], nS)
            O = alg1_star_inverse(tabs, F[0], F[1], F[2], mesh.lam)
            dui = star_values_from_planes(j, O)
        else:
            Hi = cond.Hhat[np.ix_(pos, pos)]
            dui = np.linalg.solve(Hi, r[pos])
        du[pos] += star_weights(mesh, cond.B, c, pos) * dui
    return du


# --------------------------------------------------------------------------
# Element-centred blocks (Sec. 3.4): the 3x3x3 element block around each element
# --------------------------------------------------------------------------

def eblock_centres(mesh):
    """One block per element (c1, c2, c3), x1 fastest."""
    return [(c1, c2, c3) for c3 in range(mesh.n[2]) for c2 in range(mesh.n[1]) for c1 in range(mesh.n[0])]


def eblock_check(mesh):
    """The block of element c spans elements c-1, c, c+1 along every axis (full overlap); on a periodic
    axis these must be three different elements."""
    for d in range(3):
        if mesh.periodic(d) and mesh.n[d] < 3:
            raise ValueError("element-centred blocks need at least three elements along a periodic axis")


def eblock_offsets(mesh, g, c, d):
    """Offset j of global node indices g inside the block of centre c along axis d: the block's nodes are
    (c-1) p < g < (c+2) p, j = g - (c-1) p in 1 .. 3p-1 (on a periodic axis, of the image in that range);
    returns j, or 0 where g is outside."""
    p = mesh.p
    j = np.asarray(g) - (c - 1) * p
    if mesh.periodic(d):
        j = np.mod(j, mesh.n[d] * p)
    return np.where((j >= 1) & (j <= 3 * p - 1), j, 0)


def eblock_positions(mesh, B, c):
    """Positions in the condensed vector of the nodes strictly inside the block of element c, and their
    offsets (j1, j2, j3), each in 1 .. 3p-1."""
    g1 = B % mesh.N[0]
    g2 = (B // mesh.N[0]) % mesh.N[1]
    g3 = B // (mesh.N[0] * mesh.N[1])
    j = np.stack([eblock_offsets(mesh, g, c[d], d) for d, g in enumerate((g1, g2, g3))], axis=1)
    pos = np.flatnonzero(np.all(j > 0, axis=1))
    return pos, j[pos]


def eblock_line_table(mesh, d, c):
    """1D eigen-table of the block line of element c along axis d (Sec. 3.4 with the padding of Sec. 3.3).

    Block nodes g = (c-1) p + j, j = 1 .. 3p-1 (n_S = 3p - 1): the assembled 1D matrices restricted to them
    are those of the three elements c-1, c, c+1 with the block ends removed.  Nodes that are not unknowns
    of the domain (ghost elements beyond a face, Dirichlet faces) are decoupled: S padded with identity,
    Lambda with 1.  Returns S with S^T M S = I and S^T L S = Lambda on the active nodes, Lambda, active mask.
    """
    p = mesh.p
    nS = 3 * p - 1
    Mg, Lg = assembled_1d(mesh, d)
    graw = (c - 1) * p + np.arange(1, 3 * p)
    lo, hi = mesh.g_range(d)
    if mesh.periodic(d):
        g = mesh.wrap(graw, d)
        active = np.ones(nS, bool)
    else:
        g = graw
        active = (g >= lo) & (g <= hi)
    S = np.eye(nS)
    lam = np.ones(nS)
    ia = np.flatnonzero(active)
    if ia.size:
        ga = g[ia]
        ev, V = sla.eigh(Lg[np.ix_(ga, ga)], Mg[np.ix_(ga, ga)])
        S[np.ix_(ia, ia)] = V
        lam[ia] = ev
    return S, lam, active


def eblock_count_1d(mesh, d):
    """Per global node index along axis d: the number of element-centred blocks whose node range holds it."""
    g = np.arange(mesh.N[d])
    return sum((eblock_offsets(mesh, g, c, d) > 0).astype(int) for c in range(mesh.n[d]))


def eblock_weight_1d(mesh, d, c, j, kind):
    """1D factor of the weight W_c of block c at line offsets j (1 .. 3p-1) along axis d.

    kind "element": one on the element's own nodes and zero on the other elements' (the element-centred
    counterpart of the star weights, which are one on their vertex and zero on every other vertex,
    Sec. 3.2), so a node on one of its faces, shared with the neighbour's block, takes one half (one where
    no neighbour block exists beyond a domain face).
    kind "multiplicity": the inverse number of blocks holding the node (Sec. 2.3)."""
    p = mesh.p
    j = np.asarray(j)
    if kind == "multiplicity":
        g = (c - 1) * p + j
        if mesh.periodic(d):
            g = np.mod(g, mesh.n[d] * p)
        g = np.clip(g, 0, mesh.N[d] - 1)
        return 1.0 / np.maximum(eblock_count_1d(mesh, d)[g], 1)
    if kind != "element":
        raise ValueError("kind: 'element' or 'multiplicity'")
    lo_shared = c > 0 or mesh.periodic(d)
    hi_shared = c < mesh.n[d] - 1 or mesh.periodic(d)
    w = np.where((j > p) & (j < 2 * p), 1.0, 0.0)
    w = np.where(j == p, 0.5 if lo_shared else 1.0, w)
    return np.where(j == 2 * p, 0.5 if hi_shared else 1.0, w)


def eblock_weights(mesh, B, pos, c, kind="element"):
    """W_c at the condensed positions pos of block c: the product of the 1D factors."""
    g = (B[pos] % mesh.N[0], (B[pos] // mesh.N[0]) % mesh.N[1], B[pos] // (mesh.N[0] * mesh.N[1]))
    W = np.ones(len(pos))
    for d in range(3):
        W *= eblock_weight_1d(mesh, d, c[d], eblock_offsets(mesh, g[d], c[d], d), kind)
    return W


def smoother_eblock_dense(mesh, cond, r, kind="element"):
    """Element-centred Schwarz smoother (Sec. 3.4 as a drop-in for the stars in eq. smoother_definition):
    Delta u = sum_c R_c^T W_c Hhat_c^{-1} R_c r over all elements c, Hhat_c = R_c Hhat R_c^T, W_c of the
    given kind (eblock_weight_1d); each block inverse applied densely."""
    eblock_check(mesh)
    du = np.zeros_like(r)
    for c in eblock_centres(mesh):
        pos, _ = eblock_positions(mesh, cond.B, c)
        if pos.size == 0:
            continue
        dui = np.linalg.solve(cond.Hhat[np.ix_(pos, pos)], r[pos])
        du[pos] += eblock_weights(mesh, cond.B, pos, c, kind) * dui
    return du


# --------------------------------------------------------------------------
# p-multigrid (Sec. 4.1)
# --------------------------------------------------------------------------

def level_degrees(p, p0=1):
    """p_l = p0 2^l for 0 <= l < L, p_L = p (Sec. 4.1); L smallest with p0 2^L >= p."""
    if p < p0:
        raise ValueError("p must be >= p0")
    degs = [p0]
    while degs[-1] * 2 < p:
        degs.append(degs[-1] * 2)
    if degs[-1] != p:
        degs.append(p)
    return degs


def prolongation(mesh_c, mesh_f, B_c, B_f):
    """Embedded interpolation restricted to the condensed system (Sec. 4.1).

    Built from the 3D definition: inside each element the fine nodal values are
    (J (x) J (x) J) applied to the coarse element values, J[i, j] = l^c_j(xi^f_i).
    Rows are fine free skeleton nodes, columns coarse free skeleton nodes.  GLL
    contains the element end points, so a fine skeleton node depends on coarse
    skeleton values only; that is asserted.
    """
    pc, pf = mesh_c.p, mesh_f.p
    xc, _ = gll(pc)
    xf, _ = gll(pf)
    J = interp_matrix(xc, xf)
    J3 = np.kron(J, np.kron(J, J))
    Nf = int(np.prod(mesh_f.N))
    Nc = int(np.prod(mesh_c.N))
    rowpos = -np.ones(Nf, int)
    rowpos[B_f] = np.arange(len(B_f))
    colpos = -np.ones(Nc, int)
    colpos[B_c] = np.arange(len(B_c))
    Gc = index_sets(mesh_c)["G"]
    skel_c = ((Gc[0] % pc == 0) | (Gc[1] % pc == 0) | (Gc[2] % pc == 0)).ravel()
    P = sp.lil_matrix((len(B_f), len(B_c)))
    done = np.zeros(len(B_f), bool)
    for a3 in range(mesh_f.n[2]):
        for a2 in range(mesh_f.n[1]):
            for a1 in range(mesh_f.n[0]):
                gf = _element_global_index(mesh_f, a1, a2, a3)
                gc = _element_global_index(mesh_c, a1, a2, a3)
                for li, g in enumerate(gf):
                    rp = rowpos[g]
                    if rp < 0 or done[rp]:
                        continue
                    row = J3[li]
                    nz = np.flatnonzero(np.abs(row) > 0)
                    for lj in nz:
                        gcj = gc[lj]
                        if colpos[gcj] >= 0:
                            P[rp, colpos[gcj]] = row[lj]
                        else:
                            # coarse non-free node: must be Dirichlet (value 0) or
                            # an element-interior node with a zero coefficient
                            assert skel_c[gcj] or abs(row[lj]) < 1e-12
                    done[rp] = True
    return P.tocsr()


class Hierarchy:
    """Levels, condensed operators and transfers of the p-multigrid (Sec. 4.1)."""

    def __init__(self, mesh, p0=1, nu_pre=1, nu_post=1):
        self.degs = level_degrees(mesh.p, p0)
        self.meshes = [mesh.with_degree(q) for q in self.degs]
        self.conds = [Condensed(m) for m in self.meshes]
        self.P = [None] + [prolongation(self.meshes[l - 1], self.meshes[l],
                                        self.conds[l - 1].B, self.conds[l].B)
                           for l in range(1, len(self.degs))]
        self.nu_pre, self.nu_post = nu_pre, nu_post

    @property
    def L(self):
        return len(self.degs) - 1

    def smooth(self, l, r):
        return smoother_dense(self.meshes[l], self.conds[l], r)

    def coarse_solve(self, F0):
        H0 = self.conds[0].Hhat
        return sla.solve(H0, F0, assume_a="pos") if len(F0) else F0.copy()


def vcycle(hier, u, F):
    """Algorithm 3 (multigrid V-cycle for the condensed system), literally."""
    L = hier.L
    ul = [None] * (L + 1)
    Fl = [None] * (L + 1)
    ul[L] = np.array(u, float, copy=True)
    Fl[L] = np.asarray(F, float)
    for l in range(L, 0, -1):
        if l != L:
            ul[l] = np.zeros_like(Fl[l])
        for _ in range(hier.nu_pre):
            ul[l] = ul[l] + hier.smooth(l, Fl[l] - hier.conds[l].Hhat @ ul[l])
        Fl[l - 1] = hier.P[l].T @ (Fl[l] - hier.conds[l].Hhat @ ul[l])
    ul[0] = hier.coarse_solve(Fl[0])
    for l in range(1, L + 1):
        ul[l] = ul[l] + hier.P[l] @ ul[l - 1]
        for _ in range(hier.nu_post):
            ul[l] = ul[l] + hier.smooth(l, Fl[l] - hier.conds[l].Hhat @ ul[l])
    return ul[L]


def mg_solve(hier, Fhat, rtol=1e-10, maxit=50, u0=None):
    """Algorithm 4: V-cycles until ||r|| <= rtol ||r_0|| (relative, Euclidean)."""
    H = hier.conds[-1].Hhat
    u = np.zeros_like(Fhat) if u0 is None else np.array(u0, float)
    r = Fhat - H @ u
    n0 = np.linalg.norm(r)
    hist = [n0]
    it = 0
    while hist[-1] > rtol * n0 and it < maxit:
        u = vcycle(hier, u, Fhat)
        r = Fhat - H @ u
        hist.append(np.linalg.norm(r))
        it += 1
    return u, it, np.array(hist)
