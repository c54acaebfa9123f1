"""Dense-matrix multigrid operators for brute-force checks on tiny grids.

Independent of both the oracle and the CUDA library: every operator is built
as an explicit matrix from Kronecker products of 1D stencils, and red-black
Gauss-Seidel is the textbook splitting (a lower-triangular solve in red-first
ordering).  Vectors hold interior unknowns only, x fastest.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def lap(d: int, n: int) -> np.ndarray:
    """A' = sum over axes of the 1D [-1 2 -1] matrix (unscaled 5/7-point)."""
    m = n - 1
    T = 2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    I = np.eye(m)
    A = np.zeros((m ** d, m ** d))
    for ax in range(d):
        A += _kron_all([T if a == ax else I for a in range(d)])
    return A


def prolong(d: int, nc: int) -> np.ndarray:
    """Tensor-product linear interpolation, coarse interior -> fine interior."""
    n = 2 * nc
    P1 = np.zeros((n - 1, nc - 1))
    for i in range(1, n):
        for c in range(1, nc):
            if i == 2 * c:
                P1[i - 1, c - 1] = 1.0
            elif abs(i - 2 * c) == 1:
                P1[i - 1, c - 1] = 0.5
    return _kron_all([P1] * d)


def restrict(d: int, n: int) -> np.ndarray:
    """4 x full weighting (1D weights 1/4 1/2 1/4), fine -> coarse interior."""
    nc = n // 2
    R1 = np.zeros((nc - 1, n - 1))
    for c in range(1, nc):
        for i in range(1, n):
            if i == 2 * c:
                R1[c - 1, i - 1] = 0.5
            elif abs(i - 2 * c) == 1:
                R1[c - 1, i - 1] = 0.25
    return 4.0 * _kron_all([R1] * d)


def colours(d: int, n: int) -> np.ndarray:
    """0 for red (i+j(+k) even), 1 for black, interior nodes in x-fastest order."""
    r = np.arange(1, n)
    grids = np.meshgrid(*([r] * d), indexing="ij")  # slowest axis first
    return (sum(grids) % 2).reshape(-1)


def rbgs_iteration_matrix(d: int, n: int) -> np.ndarray:
    """Error propagation of one red-then-black sweep: I - M^-1 A' with M the
    lower triangle (with diagonal) of A' in red-first ordering."""
    A = lap(d, n)
    c = colours(d, n)
    perm = np.concatenate([np.where(c == 0)[0], np.where(c == 1)[0]])
    Ap = A[np.ix_(perm, perm)]
    M = np.tril(Ap)
    Sp = np.eye(len(perm)) - sla.solve_triangular(M, Ap, lower=True)
    S = np.empty_like(Sp)
    S[np.ix_(perm, perm)] = Sp
    return S


def rbgs_sweep(d: int, n: int, b: np.ndarray, u: np.ndarray) -> np.ndarray:
    """One red-then-black sweep as a triangular solve: M u_new = b - (A'-M) u."""
    A = lap(d, n)
    c = colours(d, n)
    perm = np.concatenate([np.where(c == 0)[0], np.where(c == 1)[0]])
    Ap = A[np.ix_(perm, perm)]
    M = np.tril(Ap)
    rhs = b[perm] - (Ap - M) @ u[perm]
    up = sla.solve_triangular(M, rhs, lower=True)
    out = np.empty_like(u)
    out[perm] = up
    return out


def wj_iteration_matrix(d: int, n: int, omega: float) -> np.ndarray:
    return np.eye((n - 1) ** d) - (omega / (2 * d)) * lap(d, n)


def smoother_matrix(d, n, smoother, omega, sweeps):
    S = rbgs_iteration_matrix(d, n) if smoother == 1 else wj_iteration_matrix(d, n, omega)
    return np.linalg.matrix_power(S, sweeps)


def vcycle_error_matrix(d, n, levels, smoother=1, omega=0.8, nu1=2, nu2=2,
                        coarse_sweeps=1):
    """Error propagation E of one V-cycle with `levels` grids; coarse
    iterates start from zero, the coarsest grid is solved exactly when it has
    one unknown and by `coarse_sweeps` red-black sweeps from zero otherwise."""
    A = lap(d, n)
    I = np.eye(A.shape[0])
    if levels == 1:
        return smoother_matrix(d, n, smoother, omega, nu1)
    nc = n // 2
    if levels == 2:
        Ac = lap(d, nc)
        if nc == 2:
            Bc = np.linalg.inv(Ac)
        else:
            Sc = np.linalg.matrix_power(rbgs_iteration_matrix(d, nc), coarse_sweeps)
            Bc = (np.eye(Ac.shape[0]) - Sc) @ np.linalg.inv(Ac)
    else:
        Ec = vcycle_error_matrix(d, nc, levels - 1, smoother, omega, nu1, nu2, coarse_sweeps)
        Ac = lap(d, nc)
        Bc = (np.eye(Ac.shape[0]) - Ec) @ np.linalg.inv(Ac)
    CG = I - prolong(d, nc) @ Bc @ restrict(d, n) @ A
    return (smoother_matrix(d, n, smoother, omega, nu2) @ CG
            @ smoother_matrix(d, n, smoother, omega, nu1))


def to_vec(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a[(slice(1, -1),) * a.ndim]).reshape(-1)


def from_vec(v: np.ndarray, d: int, n: int) -> np.ndarray:
    a = np.zeros((n + 1,) * d)
    a[(slice(1, -1),) * d] = v.reshape((n - 1,) * d)
    return a


def fmg_matrix(d, n, levels, smoother=1, omega=0.8, nu1=2, nu2=2, coarse_sweeps=1):
    """FMG-V as a linear map u = M b: restricted right-hand sides, exact
    one-unknown coarsest solve, then per level u_l = P u_{l+1} followed by one
    V-cycle from that guess: u_l = E_l P u_{l+1} + (I - E_l) A_l^-1 b_l."""
    A = lap(d, n)
    if levels == 1:
        E = vcycle_error_matrix(d, n, 1, smoother, omega, nu1, nu2, coarse_sweeps)
        return (np.eye(A.shape[0]) - E) @ np.linalg.inv(A)
    nc = n // 2
    if levels == 2:
        Ac = lap(d, nc)
        if nc == 2:
            Mc = np.linalg.inv(Ac)
        else:
            Sc = np.linalg.matrix_power(rbgs_iteration_matrix(d, nc), coarse_sweeps)
            Mc = (np.eye(Ac.shape[0]) - Sc) @ np.linalg.inv(Ac)
    else:
        Mc = fmg_matrix(d, nc, levels - 1, smoother, omega, nu1, nu2, coarse_sweeps)
    E = vcycle_error_matrix(d, n, levels, smoother, omega, nu1, nu2, coarse_sweeps)
    I = np.eye(A.shape[0])
    return E @ prolong(d, nc) @ Mc @ restrict(d, n) + (I - E) @ np.linalg.inv(A)


def colour_index(d: int, n: int) -> np.ndarray:
    """The paper's multi-colour index (i mod 2) + 2 (j mod 2) (+ 4 (k mod 2)) of
    the interior nodes, x-fastest order."""
    r = np.arange(1, n)
    grids = np.meshgrid(*([r] * d), indexing="ij")  # slowest axis first
    c = np.zeros_like(grids[0])
    for ax, g in enumerate(reversed(grids)):  # x first
        c = c + (2 ** ax) * (g % 2)
    return c.reshape(-1)


def mcgs_sweep(d: int, n: int, b: np.ndarray, u: np.ndarray, backward: bool) -> np.ndarray:
    """One multi-colour Gauss-Seidel sweep as a lower-triangular solve in the
    colour ordering (colours ascending; descending for backward)."""
    A = lap(d, n)
    c = colour_index(d, n)
    cols = range(2 ** d)
    if backward:
        cols = reversed(list(cols))
    perm = np.concatenate([np.where(c == k)[0] for k in cols])
    Ap = A[np.ix_(perm, perm)]
    M = np.tril(Ap)
    rhs = b[perm] - (Ap - M) @ u[perm]
    up = sla.solve_triangular(M, rhs, lower=True)
    out = np.empty_like(u)
    out[perm] = up
    return out


def prolong_diag(d: int, nc: int) -> np.ndarray:
    """Linear interpolation on the triangulation cut along the main diagonal:
    fine 2I + delta takes coarse I (delta = 0) or the mean of coarse I and
    I + delta; coarse boundary values are 0.  Coarse interior -> fine interior."""
    n = 2 * nc
    m, mc = n - 1, nc - 1
    P = np.zeros((m ** d, mc ** d))

    def cidx(c):
        if any(v < 1 or v > nc - 1 for v in c):
            return None
        return sum((c[a] - 1) * mc ** a for a in range(d))  # x fastest

    for f in np.ndindex(*([m] * d)):
        fi = [v + 1 for v in reversed(f)]  # (x, y, z)
        row = sum((fi[a] - 1) * m ** a for a in range(d))
        base = [v // 2 for v in fi]
        delta = [v % 2 for v in fi]
        if not any(delta):
            k = cidx(base)
            if k is not None:
                P[row, k] += 1.0
        else:
            for c in (base, [base[a] + delta[a] for a in range(d)]):
                k = cidx(c)
                if k is not None:
                    P[row, k] += 0.5
    return P


def restrict_simplex(d: int, n: int) -> np.ndarray:
    """The paper's restriction stencil times 4: weight 1/2^d at 2I and
    1/2^(d+1) at 2I +- delta for the 2^d - 1 nonzero delta in {0,1}^d
    (eq. Restriction2d: (2, 1, 1, 1, 1, 1, 1)/8 in 2D)."""
    nc = n // 2
    m, mc = n - 1, nc - 1
    R = np.zeros((mc ** d, m ** d))
    w0 = 1.0 / 2 ** d

    def fidx(f):
        if any(v < 1 or v > n - 1 for v in f):
            return None
        return sum((f[a] - 1) * m ** a for a in range(d))

    deltas = [dl for dl in np.ndindex(*([2] * d)) if any(dl)]
    for c in np.ndindex(*([mc] * d)):
        ci = [v + 1 for v in reversed(c)]
        row = sum((ci[a] - 1) * mc ** a for a in range(d))
        centre = [2 * v for v in ci]
        R[row, fidx(centre)] += 4.0 * w0
        for dl in deltas:
            for sgn in (1, -1):
                k = fidx([centre[a] + sgn * dl[a] for a in range(d)])
                if k is not None:
                    R[row, k] += 4.0 * 0.5 * w0
    return R
