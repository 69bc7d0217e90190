"""Multigrid and Krylov pieces for the vertex-centred scheme, in their textbook
form (oracle; test infrastructure only).

The paper preconditions BiCGStab (the Templates book, cited in Sec. 2.3)
with one geometric-multigrid V-cycle on its hierarchy of regularly refined
grids, whose convergence rate it takes to be independent of the mesh size
(Sec. 2.3).  For the vertex-centred scheme of ``oracle.henry_vc`` the grids
are vertex-nested: coarse vertex (J, I) is fine vertex (2J, 2I).  The pieces,
on the 9-point block form of the Jacobian:

* block form: ``A[j, i, dj + 1, di + 1]`` is the 2x2 block (rows = fluid,
  salt equation; columns = p, c) coupling vertex (j, i) to vertex
  (j + dj, i + di); blocks reaching outside the grid are zero.  Vectors are
  (ny + 1, nx + 1, 2).
* ``prolong``: bilinear interpolation from the coarse vertices;
  ``restrict``: its transpose (a fine balance is shared among the coarse
  vertices with the interpolation weights), so that the coarse balances are
  sums of fine ones.
* ``hierarchy``: coarse operators rediscretised - the Jacobian of the same
  scheme on the coarser grid (same tau), at the states injected onto the
  coarse vertices; coarsening stops at 2 x 1 elements.
* ``sweep``: point-block Gauss-Seidel over the vertices of one of four
  colours (i mod 2 + 2 (j mod 2)); the 9-point stencil couples diagonal
  neighbours, so two colours would not decouple.  x_v = C_v^{-1} (b_v -
  sum_{nb != v} A_nb x_nb).
* ``vcycle``: V(nu1, nu2) from x = 0: nu1 sweeps of colours 0..3; residual;
  restriction, with the coarse Dirichlet equations' entries set to 0 (the
  correction of a Dirichlet value is 0); recursion (dense solve on the
  coarsest grid); x += P x_c; nu2 sweeps of colours 3..0.
* BiCGStab is ``oracle.mg.bicgstab`` with ``apply`` of this module as its
  operator.
"""
import numpy as np

from . import henry as cc
from . import henry_vc as vc


def blocks_from_csr(Jsp, grid):
    """(ny+1, nx+1, 3, 3, 2, 2) blocks of the vertex Jacobian ``Jsp``
    (unknown index 2 v + var, v = j (nx + 1) + i)."""
    nx1 = grid.nx + 1
    C = Jsp.tocoo()
    vr, eq = np.divmod(C.row, 2)
    vcol, var = np.divmod(C.col, 2)
    j, i = np.divmod(vr, nx1)
    jc, ic = np.divmod(vcol, nx1)
    dj, di = jc - j, ic - i
    if np.any(np.abs(dj) > 1) or np.any(np.abs(di) > 1):
        raise ValueError("matrix is not a 9-point block stencil")
    A = np.zeros((grid.ny + 1, nx1, 3, 3, 2, 2))
    np.add.at(A, (j, i, dj + 1, di + 1, eq, var), C.data)
    return A


def apply(A, x):
    """y = A x."""
    ny1, nx1 = x.shape[:2]
    xp = np.zeros((ny1 + 2, nx1 + 2, 2))
    xp[1:-1, 1:-1] = x
    y = np.zeros_like(x)
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            y += np.einsum("yxij,yxj->yxi", A[:, :, dj + 1, di + 1], xp[1 + dj:1 + dj + ny1, 1 + di:1 + di + nx1])
    return y


def prolong(xc):
    """Bilinear interpolation of coarse-vertex values to the fine vertices."""
    nyc, nxc = xc.shape[0] - 1, xc.shape[1] - 1
    x = np.zeros((2 * nyc + 1, 2 * nxc + 1) + xc.shape[2:])
    x[::2, ::2] = xc
    x[::2, 1::2] = 0.5 * (xc[:, :-1] + xc[:, 1:])
    x[1::2, ::2] = 0.5 * (xc[:-1, :] + xc[1:, :])
    x[1::2, 1::2] = 0.25 * (xc[:-1, :-1] + xc[:-1, 1:] + xc[1:, :-1] + xc[1:, 1:])
    return x


def restrict(r):
    """The transpose of ``prolong``."""
    rc = r[::2, ::2].copy()
    e = 0.5 * r[::2, 1::2]
    rc[:, :-1] += e
    rc[:, 1:] += e
    e = 0.5 * r[1::2, ::2]
    rc[:-1, :] += e
    rc[1:, :] += e
    e = 0.25 * r[1::2, 1::2]
    rc[:-1, :-1] += e
    rc[:-1, 1:] += e
    rc[1:, :-1] += e
    rc[1:, 1:] += e
    return rc


def dirichlet_mask(ny1, nx1):
    """Entries whose equation is a Dirichlet condition: p and c at x = Lx,
    c at x = 0."""
    m = np.zeros((ny1, nx1, 2), dtype=bool)
    m[:, -1, :] = True
    m[:, 0, 1] = True
    return m


def coarsest_reached(grid):
    return grid.nx <= 2 or grid.ny <= 1


def hierarchy(prm, grid, coef, p, c, p_old, c_old):
    """Block operators from the finest grid down, rediscretised at the
    injected states; ``coef`` carries uniform phi and K (the three-parameter
    model)."""
    ops = []
    g = grid
    while True:
        cg = cc.Coeffs(phi=np.full((g.ny, g.nx), coef.phi[0, 0]), K=np.full((g.ny, g.nx), coef.K[0, 0]),
                       qin=coef.qin)
        ops.append(blocks_from_csr(vc.jacobian(prm, g, cg, p, c, p_old, c_old), g))
        if coarsest_reached(g):
            return ops
        g = cc.Grid(g.nx // 2, g.ny // 2, 2.0 * g.h, g.tau, g.steps)
        p, c, p_old, c_old = p[::2, ::2], c[::2, ::2], p_old[::2, ::2], c_old[::2, ::2]


def colour_of(ny1, nx1):
    J, I = np.meshgrid(np.arange(ny1), np.arange(nx1), indexing="ij")
    return (I % 2) + 2 * (J % 2)


def sweep(A, x, b, colour):
    """One point-block Gauss-Seidel pass over the vertices of ``colour``."""
    sel = colour_of(*x.shape[:2]) == colour
    C = A[:, :, 1, 1]
    off = apply(A, x) - np.einsum("yxij,yxj->yxi", C, x)
    x = x.copy()
    x[sel] = np.linalg.solve(C[sel], (b - off)[sel][..., None])[..., 0]
    return x


def dense(A):
    """The block operator as a dense matrix (unknown index 2 v + var)."""
    ny1, nx1 = A.shape[:2]
    n = 2 * ny1 * nx1
    M = np.zeros((n, n))
    for j in range(ny1):
        for i in range(nx1):
            r = 2 * (j * nx1 + i)
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    jj, ii = j + dj, i + di
                    if 0 <= jj < ny1 and 0 <= ii < nx1:
                        q = 2 * (jj * nx1 + ii)
                        M[r:r + 2, q:q + 2] = A[j, i, dj + 1, di + 1]
    return M


def vcycle(ops, b, nu1=2, nu2=2, k=0):
    """V(nu1, nu2) approximation of A_k^{-1} b from x = 0."""
    A = ops[k]
    if k == len(ops) - 1:
        return np.linalg.solve(dense(A), b.ravel()).reshape(b.shape)
    x = np.zeros_like(b)
    for _ in range(nu1):
        for col in (0, 1, 2, 3):
            x = sweep(A, x, b, col)
    rc = restrict(b - apply(A, x))
    rc[dirichlet_mask(*rc.shape[:2])] = 0.0
    x = x + prolong(vcycle(ops, rc, nu1, nu2, k + 1))
    for _ in range(nu2):
        for col in (3, 2, 1, 0):
            x = sweep(A, x, b, col)
    return x
