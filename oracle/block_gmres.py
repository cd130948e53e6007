"""Block flexible GMRES, right-preconditioned -- oracle, test infrastructure only.

Section 6.3 solves the 32 transmitter systems of one ring together with a
pseudo-block GMRES: one Krylov space per right-hand side, with the operator
applications and dot products of all columns fused.  Section 7 names block
methods -- one Krylov space shared by all right-hand sides, which may need
fewer iterations -- as a next step.  This module states block GMRES by its
definition, for a block B of m right-hand sides and a preconditioner M:

  R_0 = B - A X_0 = V_1 S_0                       (thin QR, V_1 n x m)
  step j:  Z_j = M V_j,  W = A Z_j,
           H_ij = V_i^H W and W <- W - V_i H_ij    (i <= j, classical Gram-Schmidt, twice)
           W = V_{j+1} H_{j+1,j}                   (thin QR)
  so that A [Z_1 .. Z_k] = [V_1 .. V_{k+1}] Hbar_k (block Arnoldi relation), and
  X_k = X_0 + [Z_1 .. Z_k] Y_k,  Y_k = argmin_Y || E_1 S_0 - Hbar_k Y ||_F.

The Frobenius norm separates by column, so column c of X_k - X_0 is the
element of span[Z_1 .. Z_k] with the least residual for b_c: with a fixed M
that span is M K_k(A M, R_0), which contains each column's own space
M K_k(A M, r_0c); block GMRES therefore never ends a step with a larger
residual on any column than single-vector GMRES after the same number of steps.

The least-squares problem is solved here with a library least-squares routine
on the whole Hbar_k, not with the rotations a production solver updates.

It also states the initial guess taken from a recycled subspace (the previous
system's solutions), the recycling Section 7 cites.

Parity status: pinned by tests/test_oracle_block_gmres.py (the iterate equals
the least-residual element of the explicitly built block Krylov space, column
by column; exact solution once the space is the whole space; no column worse
than single-vector GMRES at the same step; the recycled initial guess leaves a
residual orthogonal to A span(Xprev), beats every other element of the span
tried, and is exact when Xprev holds the solution).
"""

import numpy as np


def _apply(op, X):
    if callable(op):
        return np.asarray(op(X), dtype=np.complex128)
    return np.asarray(op @ X, dtype=np.complex128)


def block_fgmres(A, B, precond=None, steps=10, rtol=0.0, X0=None):
    """Run at most `steps` block Arnoldi steps (no restart).

    A, precond: matrices or callables on [n, m] arrays (precond None = identity).
    Stops early when every column's least-squares residual is <= rtol ||b_c||.
    Returns X_k, the per-step residual norms per column (list of [m] arrays,
    from the least-squares problem), and the number of steps taken.
    """
    B = np.asarray(B, dtype=np.complex128)
    n, m = B.shape
    X0 = np.zeros_like(B) if X0 is None else np.asarray(X0, dtype=np.complex128)
    M = (lambda X: X) if precond is None else precond
    R0 = B - _apply(A, X0)
    V1, S0 = np.linalg.qr(R0)
    Vs, Zs = [V1], []
    H = np.zeros((0, 0), dtype=np.complex128)
    bnorm = np.linalg.norm(B, axis=0)
    hist = []
    Y = np.zeros((0, m), dtype=np.complex128)
    for j in range(steps):
        Zj = _apply(M, Vs[j])
        Zs.append(Zj)
        W = _apply(A, Zj)
        Vall = np.hstack(Vs)
        coef = np.zeros((Vall.shape[1], m), dtype=np.complex128)
        for _ in range(2):
            c = Vall.conj().T @ W
            W = W - Vall @ c
            coef += c
        Vn, Hn = np.linalg.qr(W)
        Vs.append(Vn)
        # Hbar_j: ((j + 2) m) x ((j + 1) m)
        Hb = np.zeros(((j + 2) * m, (j + 1) * m), dtype=np.complex128)
        Hb[: H.shape[0], : H.shape[1]] = H
        Hb[: (j + 1) * m, j * m:] = coef
        Hb[(j + 1) * m:, j * m:] = Hn
        H = Hb
        E1S0 = np.zeros(((j + 2) * m, m), dtype=np.complex128)
        E1S0[:m] = S0
        Y = np.linalg.lstsq(H, E1S0, rcond=None)[0]
        res = np.linalg.norm(E1S0 - H @ Y, axis=0)
        hist.append(res)
        if rtol > 0 and np.all(res <= rtol * bnorm):
            break
    X = X0 + np.hstack(Zs) @ Y
    return X, hist, len(Zs)


def least_residual(A, R0, basis):
    """Column by column, the least ||r_0c - A d|| over d in span(basis) (explicit least squares)."""
    AB = _apply(A, basis)
    out = np.zeros(R0.shape[1])
    for c in range(R0.shape[1]):
        y = np.linalg.lstsq(AB, R0[:, c], rcond=None)[0]
        out[c] = np.linalg.norm(R0[:, c] - AB @ y)
    return out


def krylov_basis(A, M, R0, k, block=True):
    """Columns spanning M K_k(A M, R0) (block) or, per column c, M K_k(A M, r_0c)
    (block=False returns a list of bases), built by repeated application with a
    QR at each power for conditioning."""
    Mop = (lambda X: X) if M is None else M
    if block:
        cols = []
        P = np.linalg.qr(R0)[0]
        for _ in range(k):
            Z = _apply(Mop, P)
            cols.append(Z)
            P = np.linalg.qr(_apply(A, Z))[0]
        return np.hstack(cols)
    out = []
    for c in range(R0.shape[1]):
        cols = []
        p = R0[:, c:c + 1] / np.linalg.norm(R0[:, c])
        for _ in range(k):
            z = _apply(Mop, p)
            cols.append(z)
            w = _apply(A, z)
            p = w / np.linalg.norm(w)
        out.append(np.hstack(cols))
    return out


def recycled_initial_guess(A, B, Xprev):
    """Initial guess from a recycled subspace (the recycling of Section 7,
    Parks et al.): column by column the element of span(Xprev) with the least
    residual, x0_c = Xprev y_c with y_c = argmin ||b_c - A Xprev y||.  Xprev is
    the solution block of a previous, nearby system (the previous L-BFGS step)."""
    AX = _apply(A, np.asarray(Xprev, dtype=np.complex128))
    Y = np.linalg.lstsq(AX, np.asarray(B, dtype=np.complex128), rcond=None)[0]
    return np.asarray(Xprev, dtype=np.complex128) @ Y
