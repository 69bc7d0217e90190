"""Multigrid and Krylov pieces in their textbook form (oracle; test infrastructure only).

The paper solves every Newton system with BiCGStab (the Templates book,
cited in Sec. 2.3) preconditioned by one geometric-multigrid V-cycle on the
hierarchy of regularly refined grids (Sec. 2.3); its smoother (ILU_beta) and
coarse solver (Gaussian elimination) belong to the ug4 toolbox it used.  The
GPU path keeps the V-cycle and BiCGStab and replaces the smoother by
red-black point-block Gauss-Seidel.  This module writes each of those pieces
out plainly, on the block form of the Jacobian, so that the CUDA kernels can
be compared with them one by one.

Block form: ``A[iy, ix, k]`` is the 2x2 block (rows = equations mass/salt,
columns = unknowns p/c) coupling cell (ix, iy) to its neighbour k, with
k = 0 centre, 1 west, 2 east, 3 south, 4 north; blocks across the domain
boundary are zero.  Vectors are (ny, nx, 2).

Pieces:
* ``blocks_from_csr`` - regroup the oracle's sparse Jacobian into that form.
* ``apply``           - y = A x.
* ``galerkin``        - A_c = R A P with P piecewise constant over 2x2 cells
  and R = P^T.
* ``rediscretised_hierarchy`` - coarse operators as the Jacobian of the same
  finite-volume scheme on the 2x coarser grid, evaluated at the
  cell-averaged state (coefficients averaged likewise), all scaled by the
  finest level's residual scale; coarsening stops at 2 x 1 cells.
* ``rb_sweep``        - one point-block Gauss-Seidel half-sweep over the cells
  of one colour ((ix + iy) % 2): x_P = C_P^{-1} (b_P - sum_nb A_nb x_nb).
* ``vcycle``          - V(nu1, nu2): from x = 0, nu1 x (red, black) sweeps;
  r = b - A x restricted by summation over 2x2 children; recurse (dense solve
  on 2 x 1); x += P x_c; nu2 x (red, black) sweeps.
* ``bicgstab``        - right-preconditioned BiCGStab from x = 0, stopping
  when ||r||_2 <= rtol ||b||_2.
"""
import numpy as np

from . import henry

NB_OFFSETS = {(0, 0): 0, (0, -1): 1, (0, 1): 2, (-1, 0): 3, (1, 0): 4}


def blocks_from_csr(J, nx, ny):
    """(ny, nx, 5, 2, 2) block stencil of a CSR Jacobian with 5-point structure."""
    A = np.zeros((ny, nx, 5, 2, 2))
    C = J.tocoo()
    P, eq = np.divmod(C.row, 2)
    Q, var = np.divmod(C.col, 2)
    iy, ix = np.divmod(P, nx)
    jy, jx = np.divmod(Q, nx)
    k = np.full(P.shape, -1)
    for (dy, dx), kk in NB_OFFSETS.items():
        k[(jy - iy == dy) & (jx - ix == dx)] = kk
    if np.any(k < 0):
        raise ValueError("matrix is not a 5-point block stencil")
    np.add.at(A, (iy, ix, k, eq, var), C.data)
    return A


def apply(A, x):
    """y = A x for the block stencil A and x of shape (ny, nx, 2)."""
    y = np.einsum('yxij,yxj->yxi', A[:, :, 0], x)
    y[:, 1:] += np.einsum('yxij,yxj->yxi', A[:, 1:, 1], x[:, :-1])
    y[:, :-1] += np.einsum('yxij,yxj->yxi', A[:, :-1, 2], x[:, 1:])
    y[1:, :] += np.einsum('yxij,yxj->yxi', A[1:, :, 3], x[:-1, :])
    y[:-1, :] += np.einsum('yxij,yxj->yxi', A[:-1, :, 4], x[1:, :])
    return y


def galerkin(A):
    """R A P for piecewise-constant P over 2x2 children (R = P^T): sums the
    children's blocks; couplings between two children of the same coarse cell
    land in the coarse centre block."""
    a, b = A[0::2, 0::2], A[0::2, 1::2]   # bottom-left, bottom-right child
    c, d = A[1::2, 0::2], A[1::2, 1::2]   # top-left, top-right child
    Ac = np.zeros((A.shape[0] // 2, A.shape[1] // 2, 5, 2, 2))
    Ac[:, :, 0] = (a[:, :, 0] + b[:, :, 0] + c[:, :, 0] + d[:, :, 0]
                   + a[:, :, 2] + b[:, :, 1] + c[:, :, 2] + d[:, :, 1]
                   + a[:, :, 4] + c[:, :, 3] + b[:, :, 4] + d[:, :, 3])
    Ac[:, :, 1] = a[:, :, 1] + c[:, :, 1]
    Ac[:, :, 2] = b[:, :, 2] + d[:, :, 2]
    Ac[:, :, 3] = a[:, :, 3] + b[:, :, 3]
    Ac[:, :, 4] = c[:, :, 4] + d[:, :, 4]
    return Ac


def average_children(f):
    return 0.25 * (f[0::2, 0::2] + f[0::2, 1::2] + f[1::2, 0::2] + f[1::2, 1::2])


def restrict_sum(r):
    return r[0::2, 0::2] + r[0::2, 1::2] + r[1::2, 0::2] + r[1::2, 1::2]


def prolong(xc):
    return np.repeat(np.repeat(xc, 2, axis=0), 2, axis=1)


def coarsest_reached(nx, ny):
    return nx <= 2 or ny <= 1


def rediscretised_hierarchy(prm, grid, coef, p, c, p_old, c_old):
    """Block operators of every level, finest first, scaled by the finest
    level's residual scale rho0 h^2 / tau."""
    s = henry.residual_scale(prm, grid)
    ops = []
    g, P, Cc, Po, Co, cf = grid, p, c, p_old, c_old, coef
    while True:
        J = henry.jacobian(prm, g, cf, P, Cc, Po, Co)
        ops.append(blocks_from_csr(J, g.nx, g.ny) / s)
        if coarsest_reached(g.nx, g.ny):
            return ops
        g = henry.Grid(nx=g.nx // 2, ny=g.ny // 2, h=2.0 * g.h, tau=g.tau, steps=g.steps)
        P, Cc = average_children(P), average_children(Cc)
        Po, Co = average_children(Po), average_children(Co)
        cf = henry.Coeffs(phi=average_children(cf.phi), K=average_children(cf.K), qin=cf.qin)


def galerkin_hierarchy(A0):
    ops = [A0]
    while not coarsest_reached(ops[-1].shape[1], ops[-1].shape[0]):
        ops.append(galerkin(ops[-1]))
    return ops


def dense(A):
    """Dense matrix of a block stencil (unknown index 2*(iy*nx+ix)+var)."""
    ny, nx = A.shape[:2]
    n = 2 * nx * ny
    M = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        M[:, i] = apply(A, e.reshape(ny, nx, 2)).ravel()
    return M


def rb_sweep(A, x, b, colour):
    """Point-block Gauss-Seidel over the cells of one colour, in place."""
    ny, nx = A.shape[:2]
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing='ij')
    mask = ((ix + iy) & 1) == colour
    off = apply(A, x) - np.einsum('yxij,yxj->yxi', A[:, :, 0], x)
    xn = np.linalg.solve(A[:, :, 0], (b - off)[..., None])[..., 0]
    x[mask] = xn[mask]
    return x


def vcycle(ops, b, nu1=2, nu2=2, k=0):
    """One V(nu1, nu2) cycle for A_k x = b from x = 0."""
    A = ops[k]
    if k == len(ops) - 1:
        return np.linalg.solve(dense(A), b.ravel()).reshape(b.shape)
    x = np.zeros_like(b)
    for _ in range(nu1):
        rb_sweep(A, x, b, 0)
        rb_sweep(A, x, b, 1)
    r = b - apply(A, x)
    xc = vcycle(ops, restrict_sum(r), nu1, nu2, k + 1)
    x = x + prolong(xc)
    for _ in range(nu2):
        rb_sweep(A, x, b, 0)
        rb_sweep(A, x, b, 1)
    return x


def bicgstab(A, b, precond, rtol, maxit=500):
    """Right-preconditioned BiCGStab (Templates book, Sec. 2.3.8, with the
    preconditioner applied on the right) from x = 0 with shadow residual
    r_hat = b.  ``A``: a block stencil of this module, or any callable
    z -> A z.  Returns (x, iterations, converged)."""
    matvec = A if callable(A) else (lambda z: apply(A, z))
    x = np.zeros_like(b)
    r = b.copy()
    rh = b.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, True
    rho_prev = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = np.vdot(rh, r)
        beta = (rho / rho_prev) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = precond(p)
        v = matvec(ph)
        alpha = rho / np.vdot(rh, v)
        s = r - alpha * v
        sh = precond(s)
        t = matvec(sh)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho_prev = rho
        if np.linalg.norm(r) <= rtol * nb:
            return x, it, True
    return x, maxit, False
