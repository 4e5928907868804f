"""FP64 CPU oracle for the statically condensed spectral-element p-multigrid solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, links or runs anything in this package; only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` use it.  It shares no code, tables or helpers with the CUDA path.

Modules
-------
gll       1D Gauss-Lobatto-Legendre basis: nodes, weights, differentiation and
          interpolation matrices, standard-element mass and stiffness (Sec. 2.1).
dense     O1: the plain definitions with explicit (sparse/dense) matrices on tiny
          meshes -- element assembly (Sec. 2.1), Schur complement (Sec. 2.2),
          dense star inverses (Sec. 2.3), Algorithm 1 with explicit tables,
          Algorithm 2, element-centred block inverses (Sec. 3.4),
          embedded-interpolation transfers, Algorithms 3 and 4, boundary
          kinds (Sec. 3.3) and inhomogeneous Dirichlet data by lifting (Sec. 5.2).
matfree   O2: the same steps matrix-free on nodal arrays, written as loops over
          elements and stars with per-element tensor-product operators, for
          meshes too large for O1.  Pinned against O1 by the tests.

Every function cites the section, equation or algorithm of the paper
(Huismann, Stiller, Froehlich, "Scaling to the stars -- a linearly scaling
elliptic solver for p-multigrid", arXiv:1808.03595) it follows.
"""
