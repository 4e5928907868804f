"""O2: matrix-free FP64 oracle on nodal arrays -- test infrastructure only.

Same mathematics as ``oracle.dense`` (O1), applied without global matrices so that
it reaches the mesh sizes of the benchmark workloads.  Vectors live on the global
GLL grid as nodal arrays u[g3, g2, g1]; a condensed vector is a nodal array that
is zero at element-interior nodes and on the Dirichlet boundary.

Operators follow the definitions directly and make no attempt at the paper's
O(p^3) factorisations except where the paper prescribes them (Algorithm 1):
  * element operator: eq. helmholtzop applied in tensor-product form, O(p^4);
  * condensed element operator (Sec. 2.2): Hhat_e u_B =
        (H_e [u_B; 0])_B - (H_e [0; H_II^{-1} (H_e [u_B; 0])_I])_B,
    with H_II^{-1} by 3D fast diagonalisation of the element interior block
    (eq. fast_diagonalization for one element);
  * smoother: Algorithm 2 around Algorithm 1 on every vertex star; or the
    element-centred 3^3-element blocks of Sec. 3.4, each inverted by the
    embedding of Sec. 3.1 and the full block's fast diagonalisation, weighted
    with the inverse multiplicity;
  * transfers: per-element 3D embedded interpolation and its exact transpose;
  * coarse solve: exact sparse direct solve of the full coarse system with the
    embedded right-hand side (F_hat, 0) (Sec. 3.1, eq. star_right_hand_side_full
    argument applied to the whole domain);
  * Algorithms 3 and 4 literally; Algorithm 5 (Krylov acceleration) with the
    V-cycle as preconditioner; optionally the varied smoothing counts
    nu_l = 2^(L-l) of Sec. 4.1.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla
from numpy.lib.stride_tricks import as_strided

from . import dense
from .gll import gll, interp_matrix, standard_matrices, weight_poly


# --------------------------------------------------------------------------
# element blocks of a nodal array
# --------------------------------------------------------------------------

def elem_view(u, mesh):
    """Overlapping view (n3, n2, n1, p+1, p+1, p+1) of the element blocks of a nodal array."""
    p = mesh.p
    n1, n2, n3 = mesh.n
    s3, s2, s1 = u.strides
    return as_strided(u, shape=(n3, n2, n1, p + 1, p + 1, p + 1),
                      strides=(p * s3, p * s2, p * s1, s3, s2, s1), writeable=False)


def elem_blocks(u, mesh):
    """Element blocks of a nodal array; periodic images take the value of their unknown."""
    return np.array(elem_view(np.ascontiguousarray(dense.sync_images(mesh, u), dtype=float), mesh))


def _fold_images(out, mesh):
    """Periodic axes: add the image plane into the first plane, then copy it back."""
    for d in range(3):
        if mesh.periodic(d):
            ax = 2 - d
            idx0 = [slice(None)] * 3
            idx1 = [slice(None)] * 3
            idx0[ax] = 0
            idx1[ax] = out.shape[ax] - 1
            out[tuple(idx0)] += out[tuple(idx1)]
    return dense.sync_images(mesh, out)


def assemble_blocks(blocks, mesh):
    """Sum element blocks into a nodal array (direct stiffness summation)."""
    out = np.zeros(mesh.shape)
    p = mesh.p
    n1, n2, n3 = mesh.n
    s3, s2, s1 = out.strides
    view = as_strided(out, shape=(n3, n2, n1, p + 1, p + 1, p + 1),
                      strides=(p * s3, p * s2, p * s1, s3, s2, s1), writeable=True)
    # elements of one parity class share no node, so each class is one vectorised add
    for q3 in (0, 1):
        for q2 in (0, 1):
            for q1 in (0, 1):
                view[q3::2, q2::2, q1::2] += blocks[q3::2, q2::2, q1::2]
    return _fold_images(out, mesh)


def masks(mesh):
    """Boolean nodal masks: skeleton (element boundaries) and free (not on a Dirichlet face)."""
    p = mesh.p
    G = np.meshgrid(np.arange(mesh.N[2]), np.arange(mesh.N[1]), np.arange(mesh.N[0]), indexing="ij")
    g3, g2, g1 = G
    skel = (g1 % p == 0) | (g2 % p == 0) | (g3 % p == 0)
    free = np.ones(mesh.shape, bool)
    for d, g in enumerate((g1, g2, g3)):
        lo, hi = mesh.g_range(d)
        free &= (g >= lo) & (g <= hi)
    return skel, free


def condensed_mask(mesh):
    skel, free = masks(mesh)
    return skel & free


def elem_coeffs(mesh):
    """d_e = h1 h2 h3 / 8 (lambda, 4/h1^2, 4/h2^2, 4/h3^2) for every element (Sec. 2.1)."""
    h3, h2, h1 = np.meshgrid(mesh.h[2], mesh.h[1], mesh.h[0], indexing="ij")
    vol = h1 * h2 * h3 / 8.0
    return np.stack([vol * mesh.lam, vol * 4.0 / h1**2, vol * 4.0 / h2**2, vol * 4.0 / h3**2], axis=-1)


def apply_elem_op(X, d, p):
    """eq. helmholtzop on element blocks X[..., i3, i2, i1] with coefficients d[..., 4]."""
    M, L = standard_matrices(p)
    w = np.diag(M)
    W3, W2, W1 = w[:, None, None], w[None, :, None], w[None, None, :]
    t0 = X * (W3 * W2 * W1)
    t1 = np.einsum("...ijk,ck->...ijc", X, L) * (W3 * W2)
    t2 = np.einsum("...ijk,bj->...ibk", X, L) * (W3 * W1)
    t3 = np.einsum("...ijk,ai->...ajk", X, L) * (W2 * W1)
    e = (Ellipsis, None, None, None)
    return d[..., 0][e] * t0 + d[..., 1][e] * t1 + d[..., 2][e] * t2 + d[..., 3][e] * t3


def interior_eigen(p):
    """Reference interior generalized eigenpairs S^T L_II S = Lambda, S^T M_II S = I (Sec. 3.2)."""
    M, L = standard_matrices(p)
    lam, S = sla.eigh(L[1:p, 1:p], M[1:p, 1:p])
    return S, lam


def hii_inv(Y, d, p):
    """H_II^{-1} on interior blocks Y[..., m, m, m] by fast diagonalisation (eq. fast_diagonalization)."""
    S, lam = interior_eigen(p)
    Z = np.einsum("...ijk,ia,jb,kc->...abc", Y, S, S, S, optimize=True)
    D = (d[..., 0][..., None, None, None]
         + d[..., 3][..., None, None, None] * lam[:, None, None]
         + d[..., 2][..., None, None, None] * lam[None, :, None]
         + d[..., 1][..., None, None, None] * lam[None, None, :])
    Z = Z / D
    return np.einsum("...abc,ia,jb,kc->...ijk", Z, S, S, S, optimize=True)


def _interior(X):
    return X[..., 1:-1, 1:-1, 1:-1]


def _zero_interior(X):
    Y = X.copy()
    Y[..., 1:-1, 1:-1, 1:-1] = 0.0
    return Y


def _only_interior(Xi, p):
    shp = Xi.shape[:-3] + (p + 1, p + 1, p + 1)
    Y = np.zeros(shp)
    Y[..., 1:-1, 1:-1, 1:-1] = Xi
    return Y


# --------------------------------------------------------------------------
# condensed operator, condensation, recovery (Sec. 2.2; Algorithm 4 first/last lines)
# --------------------------------------------------------------------------

def apply_condensed(mesh, u, chunk=512):
    """y = Hhat u for a condensed nodal array u (element by element, then assembled)."""
    p = mesh.p
    u = np.where(condensed_mask(mesh), u, 0.0)
    blocks = elem_blocks(u, mesh)
    d = elem_coeffs(mesh)
    n1, n2, n3 = mesh.n
    bflat = blocks.reshape(-1, p + 1, p + 1, p + 1)
    dflat = d.reshape(-1, 4)
    out = np.empty_like(bflat)
    for s in range(0, bflat.shape[0], chunk):
        X = bflat[s:s + chunk]
        dd = dflat[s:s + chunk]
        t = apply_elem_op(X, dd, p)
        if p > 1:
            xi = hii_inv(_interior(t), dd, p)
            t = t - apply_elem_op(_only_interior(xi, p), dd, p)
        out[s:s + chunk] = _zero_interior(t)
    y = assemble_blocks(out.reshape(n3, n2, n1, p + 1, p + 1, p + 1), mesh)
    return np.where(condensed_mask(mesh), y, 0.0)


def mass_diag(mesh):
    """Assembled diagonal GLL mass: element mass (h1 h2 h3 / 8) M (x) M (x) M summed (Sec. 2.1)."""
    _, w = gll(mesh.p)
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    h3, h2, h1 = np.meshgrid(mesh.h[2], mesh.h[1], mesh.h[0], indexing="ij")
    blocks = (h1 * h2 * h3 / 8.0)[..., None, None, None] * W
    return assemble_blocks(blocks, mesh)


def apply_full(mesh, u, chunk=512):
    """H u on every node of a nodal array (eq. helmholtzop per element, assembled), periodic images synced."""
    p = mesh.p
    d = elem_coeffs(mesh)
    n1, n2, n3 = mesh.n
    bflat = elem_blocks(u, mesh).reshape(-1, p + 1, p + 1, p + 1)
    dflat = d.reshape(-1, 4)
    out = np.empty_like(bflat)
    for s in range(0, bflat.shape[0], chunk):
        out[s:s + chunk] = apply_elem_op(bflat[s:s + chunk], dflat[s:s + chunk], p)
    return assemble_blocks(out.reshape(n3, n2, n1, p + 1, p + 1, p + 1), mesh)


def lifted_load(mesh, f, g):
    """Load of the homogeneous problem for u = u_0 + E g (inhomogeneous Dirichlet data by lifting, the Sec. 5.2
    test problem): F = M f - H E g, E g equal to g on the Dirichlet-face nodes and zero elsewhere."""
    Eg = np.where(mesh.dirichlet_mask(), np.asarray(g, float), 0.0)
    return mass_diag(mesh) * np.asarray(f, float) - apply_full(mesh, Eg)


def condense_rhs(mesh, f, chunk=512):
    """F = M f;  Fhat = F_B - sum_e H_BI H_II^{-1} F_I (Algorithm 4, condensation step)."""
    return condense_load(mesh, mass_diag(mesh) * np.asarray(f, float), chunk)


def condense_load(mesh, F, chunk=512):
    """Fhat = F_B - sum_e H_BI H_II^{-1} F_I for an assembled nodal load F (Sec. 2.2)."""
    p = mesh.p
    F = np.asarray(F, float)
    Fh = np.where(condensed_mask(mesh), F, 0.0)
    if p == 1:
        return Fh
    d = elem_coeffs(mesh)
    blocks = elem_blocks(F, mesh)
    n1, n2, n3 = mesh.n
    bflat = blocks.reshape(-1, p + 1, p + 1, p + 1)
    dflat = d.reshape(-1, 4)
    out = np.empty_like(bflat)
    for s in range(0, bflat.shape[0], chunk):
        dd = dflat[s:s + chunk]
        xi = hii_inv(_interior(bflat[s:s + chunk]), dd, p)
        out[s:s + chunk] = _zero_interior(apply_elem_op(_only_interior(xi, p), dd, p))
    Z = assemble_blocks(out.reshape(n3, n2, n1, p + 1, p + 1, p + 1), mesh)
    return np.where(condensed_mask(mesh), Fh - Z, 0.0)


def recover(mesh, f, uhat, chunk=512):
    """Nodal u: skeleton values from uhat, u_I = H_II^{-1} (F_I - H_IB u_B) per element."""
    return recover_load(mesh, mass_diag(mesh) * np.asarray(f, float), uhat, chunk)


def recover_load(mesh, F, uhat, chunk=512):
    """recover() for an assembled nodal load F instead of M f."""
    p = mesh.p
    u = np.where(condensed_mask(mesh), uhat, 0.0)
    if p == 1:
        return dense.sync_images(mesh, u)
    F = np.asarray(F, float)
    d = elem_coeffs(mesh)
    ub = elem_blocks(u, mesh).reshape(-1, p + 1, p + 1, p + 1)
    fb = elem_blocks(F, mesh).reshape(-1, p + 1, p + 1, p + 1)
    dflat = d.reshape(-1, 4)
    n1, n2, n3 = mesh.n
    ui = np.empty((ub.shape[0], p - 1, p - 1, p - 1))
    for s in range(0, ub.shape[0], chunk):
        dd = dflat[s:s + chunk]
        t = apply_elem_op(ub[s:s + chunk], dd, p)
        ui[s:s + chunk] = hii_inv(_interior(fb[s:s + chunk]) - _interior(t), dd, p)
    out = u.copy()
    ui = ui.reshape(n3, n2, n1, p - 1, p - 1, p - 1)
    for a3 in range(n3):
        for a2 in range(n2):
            for a1 in range(n1):
                out[a3 * p + 1:(a3 + 1) * p, a2 * p + 1:(a2 + 1) * p, a1 * p + 1:(a1 + 1) * p] = ui[a3, a2, a1]
    return dense.sync_images(mesh, out)


# --------------------------------------------------------------------------
# star smoother (Algorithm 2 around Algorithm 1)
# --------------------------------------------------------------------------

class StarTables:
    """Per vertex line eigen-tables (Sec. 3.2, 3.3) and 1D weight vectors of one level."""

    def __init__(self, mesh):
        self.mesh = mesh
        p = mesh.p
        m = p - 1
        self.S, self.Lam, self.act, self.wl = [], [], [], []
        x = mesh.node_coords()
        j = np.arange(-m, m + 1)
        xi, _ = gll(p)
        for d in range(3):
            Sd, Ld, Ad, Wd = [], [], [], []
            for c in range(mesh.n[d] + (0 if mesh.periodic(d) else 1)):
                S, lam, act = dense.star_line_table(mesh, d, c)
                Sd.append(S)
                Ld.append(lam)
                Ad.append(act)
                g = c * p + j
                wv = np.zeros(len(j))
                if mesh.periodic(d):
                    # every offset lies inside the domain; t = its reference distance to the vertex
                    Wd.append(weight_poly((1.0 + xi[np.abs(j)]) / 2.0))
                    continue
                for k, gg in enumerate(g):
                    if 0 <= gg < mesh.N[d]:
                        dist = x[d][gg] - mesh.X[d][c]
                        if dist == 0.0:
                            wv[k] = 1.0
                            continue
                        side = c if dist > 0 else c - 1
                        wv[k] = weight_poly(abs(dist) / mesh.h[d][side])
                Wd.append(wv)
            self.S.append(np.array(Sd))
            self.Lam.append(np.array(Ld))
            self.act.append(np.array(Ad))
            self.wl.append(np.array(Wd))


def smooth(mesh, r, tables=None, chunk=128):
    """Delta u = Smoother(r) (Algorithm 2), each star inverted by Algorithm 1.

    Star outputs are combined as W_i times the solution; a node stored on
    several planes of one star contributes the mean of its plane values.
    """
    p = mesh.p
    m = p - 1
    nS = 2 * m + 1
    if tables is None:
        tables = StarTables(mesh)
    r = np.where(condensed_mask(mesh), r, 0.0)
    P = p  # padding so every star plane slice is in range
    rp = _pad_star(mesh, r, P)
    dup = np.zeros_like(rp)
    verts = np.array(dense.star_vertices(mesh))
    j = np.arange(-m, m + 1)
    z = (j == 0)
    mult = 1.0 + z[:, None] + z[None, :]
    lam = mesh.lam
    for s in range(0, len(verts), chunk):
        V = verts[s:s + chunk]
        c1, c2, c3 = V[:, 0], V[:, 1], V[:, 2]
        o1 = (c1 * p + P)[:, None, None]
        o2 = (c2 * p + P)[:, None, None]
        o3 = (c3 * p + P)[:, None, None]
        jj = j[None, :, None]
        kk = j[None, None, :]
        # plane gathers: F1[j2, j3], F2[j1, j3], F3[j1, j2]
        i1 = (o3 + kk, o2 + jj, o1 + 0 * jj)
        i2 = (o3 + kk, o2 + 0 * jj, o1 + jj)
        i3 = (o3 + 0 * jj, o2 + kk, o1 + jj)
        F1 = rp[i1] / mult
        F2 = rp[i2] / mult
        F3 = rp[i3] / mult
        S1, S2, S3 = tables.S[0][c1], tables.S[1][c2], tables.S[2][c3]
        L1, L2, L3 = tables.Lam[0][c1], tables.Lam[1][c2], tables.Lam[2][c3]
        s1, s2, s3 = S1[:, m, :], S2[:, m, :], S3[:, m, :]
        A1 = np.einsum("zjb,zjk,zkc->zbc", S2, F1, S3, optimize=True)
        A2 = np.einsum("zja,zjk,zkc->zac", S1, F2, S3, optimize=True)
        A3 = np.einsum("zja,zjk,zkb->zab", S1, F3, S2, optimize=True)
        E = (s1[:, :, None, None] * A1[:, None, :, :]
             + s2[:, None, :, None] * A2[:, :, None, :]
             + s3[:, None, None, :] * A3[:, :, :, None])
        D = lam + L1[:, :, None, None] + L2[:, None, :, None] + L3[:, None, None, :]
        Vv = E / D
        B1 = np.einsum("za,zabc->zbc", s1, Vv)
        B2 = np.einsum("zb,zabc->zac", s2, Vv)
        B3 = np.einsum("zc,zabc->zab", s3, Vv)
        O1 = np.einsum("zjb,zbc,zkc->zjk", S2, B1, S3, optimize=True)
        O2 = np.einsum("zja,zac,zkc->zjk", S1, B2, S3, optimize=True)
        O3 = np.einsum("zja,zab,zkb->zjk", S1, B3, S2, optimize=True)
        w1, w2, w3 = tables.wl[0][c1], tables.wl[1][c2], tables.wl[2][c3]
        a1, a2, a3 = tables.act[0][c1], tables.act[1][c2], tables.act[2][c3]
        # W/mult on each plane; masked where the node is not a star node
        W1 = (w2[:, :, None] * w3[:, None, :]) * (a1[:, m][:, None, None] & a2[:, :, None] & a3[:, None, :])
        W2 = (w1[:, :, None] * w3[:, None, :]) * (a2[:, m][:, None, None] & a1[:, :, None] & a3[:, None, :])
        W3 = (w1[:, :, None] * w2[:, None, :]) * (a3[:, m][:, None, None] & a1[:, :, None] & a2[:, None, :])
        np.add.at(dup, i1, W1 * O1 / mult)
        np.add.at(dup, i2, W2 * O2 / mult)
        np.add.at(dup, i3, W3 * O3 / mult)
    du = _unpad_star(mesh, dup, P)
    return np.where(condensed_mask(mesh), du, 0.0)


class EBlockTables:
    """Per element and axis the block line eigen-tables (Sec. 3.4) and the 1D weight factors of the blocks
    (dense.eblock_weight_1d of the given kind, at line offsets 1 .. 3p-1)."""

    def __init__(self, mesh, kind="element"):
        dense.eblock_check(mesh)
        self.mesh = mesh
        self.kind = kind
        self.S, self.Lam, self.act, self.wl = [], [], [], []
        j = np.arange(1, 3 * mesh.p)
        for d in range(3):
            tabs = [dense.eblock_line_table(mesh, d, c) for c in range(mesh.n[d])]
            self.S.append(np.array([t[0] for t in tabs]))
            self.Lam.append(np.array([t[1] for t in tabs]))
            self.act.append(np.array([t[2] for t in tabs]))
            self.wl.append(np.array([dense.eblock_weight_1d(mesh, d, c, j, kind) for c in range(mesh.n[d])]))


def smooth_eblock(mesh, r, tables=None):
    """Delta u = sum_c R_c^T W_c Hhat_c^{-1} R_c r over the element-centred blocks (Sec. 3.4).

    Each block inverse by the embedding of Sec. 3.1 and the block's fast diagonalisation: the condensed
    residual, zero at element-interior nodes, is the right-hand side of the full 3^3-element block
    problem; its solution (S3 x S2 x S1) D^{-1} (S3 x S2 x S1)^T on the block, read at the block's skeleton
    nodes, is Hhat_c^{-1} R_c r.  W_c: the tables' weights (dense.eblock_weight_1d).
    """
    p = mesh.p
    tables = tables or EBlockTables(mesh)
    r = np.where(condensed_mask(mesh), r, 0.0)
    du = np.zeros(mesh.shape)
    j = np.arange(1, 3 * p)
    on_plane = (j == p) | (j == 2 * p)
    lam = mesh.lam
    for c in dense.eblock_centres(mesh):
        gi, ok = [], []
        for d in range(3):
            g = (c[d] - 1) * p + j
            if mesh.periodic(d):
                gi.append(np.mod(g, mesh.n[d] * p))
                ok.append(np.ones(len(j), bool))
            else:
                ok.append((g >= 0) & (g < mesh.N[d]))
                gi.append(np.clip(g, 0, mesh.N[d] - 1))
        idx = np.ix_(gi[2], gi[1], gi[0])
        inside = ok[2][:, None, None] & ok[1][None, :, None] & ok[0][None, None, :]
        R = np.where(inside, r[idx], 0.0)
        S1, S2, S3 = tables.S[0][c[0]], tables.S[1][c[1]], tables.S[2][c[2]]
        Ft = np.einsum("ijk,ic,jb,ka->cba", R, S3, S2, S1, optimize=True)
        D = lam + tables.Lam[2][c[2]][:, None, None] + tables.Lam[1][c[1]][None, :, None] \
            + tables.Lam[0][c[0]][None, None, :]
        U = np.einsum("cba,ic,jb,ka->ijk", Ft / D, S3, S2, S1, optimize=True)
        skel = on_plane[:, None, None] | on_plane[None, :, None] | on_plane[None, None, :]
        W = tables.wl[2][c[2]][:, None, None] * tables.wl[1][c[1]][None, :, None] * tables.wl[0][c[0]][None, None, :]
        np.add.at(du, idx, np.where(inside & skel, W * U, 0.0))
    return np.where(condensed_mask(mesh), du, 0.0)


def _pad_star(mesh, r, P):
    """Pad a nodal array by P on every side: zeros, or on a periodic axis the
    values wrapped around the n_d p unknowns (a star near one end reads the other)."""
    for d in range(3):
        ax = 2 - d
        if mesh.periodic(d):
            Lp = mesh.n[d] * mesh.p
            core = np.take(r, np.arange(Lp), axis=ax)
            r = np.concatenate([np.take(core, np.arange(Lp - P, Lp), axis=ax), core,
                                np.take(core, np.arange(0, P + 1), axis=ax)], axis=ax)
        else:
            pad = [(0, 0)] * 3
            pad[ax] = (P, P)
            r = np.pad(r, pad)
    return r


def _unpad_star(mesh, dup, P):
    """Inverse of _pad_star for accumulated values: margins of a periodic axis
    are added to the unknowns they wrap onto, then the image plane is set."""
    for d in range(3):
        ax = 2 - d
        Np = dup.shape[ax]
        if mesh.periodic(d):
            Lp = mesh.n[d] * mesh.p
            core = np.take(dup, np.arange(P, P + Lp), axis=ax)
            left = np.take(dup, np.arange(0, P), axis=ax)            # wraps onto Lp - P .. Lp - 1
            right = np.take(dup, np.arange(P + Lp, Np), axis=ax)     # wraps onto 0 .. P
            idx = [slice(None)] * 3
            idx[ax] = slice(Lp - P, Lp)
            core[tuple(idx)] += left
            idx[ax] = slice(0, right.shape[ax])
            core[tuple(idx)] += right
            dup = np.concatenate([core, np.take(core, [0], axis=ax)], axis=ax)
        else:
            dup = np.take(dup, np.arange(P, Np - P), axis=ax)
    return dup


# --------------------------------------------------------------------------
# transfers (Sec. 4.1)
# --------------------------------------------------------------------------

def _interp(mesh_c, mesh_f):
    xc, _ = gll(mesh_c.p)
    xf, _ = gll(mesh_f.p)
    return interp_matrix(xc, xf)


def prolong(mesh_c, mesh_f, uc):
    """Fine condensed nodal array J uc: per-element (J (x) J (x) J) on the coarse skeleton values."""
    J = _interp(mesh_c, mesh_f)
    uc = np.where(condensed_mask(mesh_c), uc, 0.0)
    Xc = elem_blocks(uc, mesh_c)
    Xf = np.einsum("ai,bj,ck,...ijk->...abc", J, J, J, Xc, optimize=True)
    out = np.zeros(mesh_f.shape)
    pf = mesh_f.p
    n1, n2, n3 = mesh_f.n
    for a3 in range(n3):
        for a2 in range(n2):
            for a1 in range(n1):
                out[a3 * pf:(a3 + 1) * pf + 1, a2 * pf:(a2 + 1) * pf + 1, a1 * pf:(a1 + 1) * pf + 1] = Xf[a3, a2, a1]
    return np.where(condensed_mask(mesh_f), out, 0.0)


def multiplicity(mesh):
    """Number of elements sharing each node."""
    one = np.ones((mesh.n[2], mesh.n[1], mesh.n[0], mesh.p + 1, mesh.p + 1, mesh.p + 1))
    return assemble_blocks(one, mesh)


def restrict(mesh_f, mesh_c, rf):
    """Exact transpose of ``prolong`` on condensed vectors."""
    J = _interp(mesh_c, mesh_f)
    rf = np.where(condensed_mask(mesh_f), rf, 0.0) / multiplicity(mesh_f)
    Xf = elem_blocks(rf, mesh_f)
    Xc = np.einsum("ai,bj,ck,...abc->...ijk", J, J, J, Xf, optimize=True)
    out = assemble_blocks(Xc, mesh_c)
    return np.where(condensed_mask(mesh_c), out, 0.0)


# --------------------------------------------------------------------------
# coarse solve, V-cycle, solver
# --------------------------------------------------------------------------

class CoarseSolver:
    """Exact coarse solve: full system at p0 with embedded right-hand side (F_hat, 0)."""

    def __init__(self, mesh):
        self.mesh = mesh
        H = dense.assemble_H(mesh)
        sets = dense.index_sets(mesh)
        self.free = sets["free"]
        self.lu = spla.splu(H[self.free][:, self.free].tocsc())

    def solve(self, Fh):
        rhs = np.where(condensed_mask(self.mesh), Fh, 0.0).ravel()[self.free]
        u = np.zeros(int(np.prod(self.mesh.N)))
        u[self.free] = self.lu.solve(rhs)
        return np.where(condensed_mask(self.mesh), u.reshape(self.mesh.shape), 0.0)


class MG:
    """p-multigrid hierarchy (Sec. 4.1) on nodal condensed arrays."""

    def __init__(self, mesh, p0=1, nu_pre=1, nu_post=1, nu_vary=False, smoother="star"):
        self.degs = dense.level_degrees(mesh.p, p0)
        self.meshes = [mesh.with_degree(q) for q in self.degs]
        kinds = {"element": "element", "element_mult": "multiplicity"}
        if smoother != "star" and smoother not in kinds:
            raise ValueError("smoother: 'star' (Algorithm 2), 'element' or 'element_mult' (element-centred "
                             "blocks of Sec. 3.4 with element or inverse-multiplicity weights)")
        self.smoother = smoother
        self.tables = [(StarTables(m) if smoother == "star" else EBlockTables(m, kinds[smoother])) if l > 0 else None
                       for l, m in enumerate(self.meshes)]
        self.coarse = CoarseSolver(self.meshes[0])
        self.nu_pre, self.nu_post = nu_pre, nu_post
        self.nu_vary = nu_vary

    @property
    def L(self):
        return len(self.degs) - 1

    def nu(self, l, base):
        """Smoothing steps on level l (Sec. 4.1): the base count, or base * 2^(L-l) when varied."""
        return base * 2 ** (self.L - l) if self.nu_vary else base

    def op(self, l, u):
        return apply_condensed(self.meshes[l], u)

    def smooth(self, l, r):
        if self.smoother != "star":
            return smooth_eblock(self.meshes[l], r, self.tables[l])
        return smooth(self.meshes[l], r, self.tables[l])


def vcycle(mg, u, F):
    """Algorithm 3, literally, on nodal condensed arrays."""
    L = mg.L
    ul = [None] * (L + 1)
    Fl = [None] * (L + 1)
    ul[L] = np.array(u, float, copy=True)
    Fl[L] = np.asarray(F, float)
    for l in range(L, 0, -1):
        if l != L:
            ul[l] = np.zeros_like(Fl[l])
        for _ in range(mg.nu(l, mg.nu_pre)):
            ul[l] = ul[l] + mg.smooth(l, Fl[l] - mg.op(l, ul[l]))
        Fl[l - 1] = restrict(mg.meshes[l], mg.meshes[l - 1], Fl[l] - mg.op(l, ul[l]))
    ul[0] = mg.coarse.solve(Fl[0])
    for l in range(1, L + 1):
        ul[l] = ul[l] + prolong(mg.meshes[l - 1], mg.meshes[l], ul[l - 1])
        for _ in range(mg.nu(l, mg.nu_post)):
            ul[l] = ul[l] + mg.smooth(l, Fl[l] - mg.op(l, ul[l]))
    return ul[L]


def mg_solve(mg, Fhat, rtol=1e-10, maxit=50):
    """Algorithm 4: condensed V-cycle iteration to ||r|| <= rtol ||r_0||; returns (u, n, history)."""
    u = np.zeros_like(Fhat)
    r = Fhat - mg.op(mg.L, u)
    n0 = np.linalg.norm(r)
    hist = [n0]
    it = 0
    while hist[-1] > rtol * n0 and it < maxit:
        u = vcycle(mg, u, Fhat)
        r = Fhat - mg.op(mg.L, u)
        hist.append(np.linalg.norm(r))
        it += 1
    return u, it, np.array(hist)


def ipcg(op, precond, b, rtol=1e-10, maxit=50):
    """Algorithm 5's iteration: inexact preconditioned CG from u = 0.

    op(v) applies the SPD operator, precond(r) the (possibly non-symmetric or
    varying) preconditioner.  beta uses the difference of the new and the old
    residual against z, so the method tolerates preconditioners that are not
    symmetric (the weighted smoother makes the V-cycle one).  Stops at
    ||r|| <= rtol ||r_0|| with the recursively updated residual.
    Returns (u, iterations, residual-norm history).
    """
    u = np.zeros_like(b)
    r = b - op(u)
    s = r.copy()          # makes beta = 0 in the first iteration
    p = np.zeros_like(b)
    delta = 1.0
    n0 = np.linalg.norm(r)
    hist = [n0]
    it = 0
    while hist[-1] > rtol * n0 and it < maxit:
        z = precond(r)
        gamma = float(np.vdot(z, r))
        gamma0 = float(np.vdot(z, s))
        beta = (gamma - gamma0) / delta
        delta = gamma
        p = beta * p + z
        q = op(p)
        alpha = gamma / float(np.vdot(q, p))
        s = r.copy()
        u = u + alpha * p
        r = r - alpha * q
        hist.append(np.linalg.norm(r))
        it += 1
    return u, it, np.array(hist)


def kmg_solve(mg, Fhat, rtol=1e-10, maxit=50):
    """Algorithm 5: Krylov-accelerated multigrid, the V-cycle MultigridCycle(0, r) as preconditioner."""
    return ipcg(lambda v: mg.op(mg.L, v), lambda r: vcycle(mg, np.zeros_like(r), r), Fhat, rtol, maxit)


def solve(mesh, f, p0=1, rtol=1e-10, maxit=50):
    """Whole solver: condense, Algorithm 4, recover.  Returns (u_nodal, iterations, history)."""
    mg = MG(mesh, p0)
    Fh = condense_rhs(mesh, f)
    uh, it, hist = mg_solve(mg, Fh, rtol, maxit)
    return recover(mesh, f, uh), it, hist


def solve_dirichlet(mesh, f, g, p0=1, rtol=1e-10, maxit=50, krylov=False, mg=None):
    """Whole solver with inhomogeneous Dirichlet data g (nodal; read on the Dirichlet faces only), by lifting:
    F = M f - H E g, condense, Algorithm 4 (or 5), recover u_0, u = u_0 + E g.
    Returns (u_nodal, iterations, history)."""
    mg = mg or MG(mesh, p0)
    F = lifted_load(mesh, f, g)
    Fh = condense_load(mesh, F)
    uh, it, hist = (kmg_solve if krylov else mg_solve)(mg, Fh, rtol, maxit)
    u = recover_load(mesh, F, uh) + np.where(mesh.dirichlet_mask(), np.asarray(g, float), 0.0)
    return u, it, hist
