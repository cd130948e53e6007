"""Direct solves, S-parameters, misfit, adjoint and gradient (Sections 4 and 5).

S-parameters (Eq. sij) with edge-current receivers: the receiver weight is
q_i = s_i e_{k_i} (unit norm), so S_ij = conj(q_i^T u_j) / |q_i|^2 =
conj(s_i u_j[k_i]).  Since A = A^T (bilinear form) S is symmetric.

Misfit (Eq. defJ): J = 1/2 sum_ij w_ij |S_ij - S^mes_ij|^2 (w = 1 in Eq. defJ).
With r = S - S^mes, dJ = Re sum_j g_j^T du_j where g_j = sum_i w_ij r_ij q_i is
the discrete adjoint source of Eq. pbadj.  The adjoint fields are
lambda_j = A^{-T} g_j = A^{-1} g_j (state and adjoint share one operator,
Section 5), and du_j = -A^{-1} dA u_j gives, per tet t,

    dJ = Re sum_t d(eps_t) G_t,
    G_t = sum_j lambda_{j,t}^T (k0^2 M_t - i k0 / (2 sqrt(eps_t)) B_t) u_{j,t},

where B_t sums the face matrices of the impedance faces owned by t (beta
depends on the owning tet's eps).  The volume term is the discrete form of
DJ = Re int conj(d kappa) sum_j conj(E_j . F_j) with kappa = k0^2 eps_r.
Returned: conj(G_t) = dJ/dRe(eps_t) + i dJ/dIm(eps_t).
"""

import numpy as np
import scipy.sparse.linalg as spla

from .assemble import assemble_system, antenna_edges, build_rhs, impedance_faces
from .constants import k0_of
from .fem import element_matrices, face_matrix


def direct_solve(A, B):
    """u = A^{-1} B by sparse LU (SuperLU, minimum degree on A^T + A)."""
    lu = spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A")
    return lu.solve(np.asarray(B, dtype=np.complex128)), lu


def s_matrix(U, rx_dofs, rx_signs):
    """S[i, j] = conj(s_i U[k_i, j])."""
    return np.conj(rx_signs[:, None] * U[rx_dofs, :])


def misfit(S, S_meas, w=None):
    r = S - S_meas
    if w is None:
        w = np.ones(S.shape)
    return 0.5 * float(np.sum(w * np.abs(r) ** 2)), r


def adjoint_rhs(ndof, r, w, rx_dofs, rx_signs):
    """g_j = sum_i w_ij r_ij s_i e_{k_i}."""
    if w is None:
        w = np.ones(r.shape)
    g = np.zeros((ndof, r.shape[1]), dtype=np.complex128)
    for i, (k, s) in enumerate(zip(rx_dofs, rx_signs)):
        g[k, :] += w[i, :] * r[i, :] * s
    return g


def gradient(xyz, topo, eps, freq, U, Lam, M=None):
    """conj(G_t) for every tet (see module docstring)."""
    eps = np.asarray(eps, dtype=np.complex128)
    k0 = k0_of(freq)
    if M is None:
        _, M = element_matrices(xyz, topo)
    n = topo.ndof
    Up = np.concatenate([U, np.zeros((1, U.shape[1]), dtype=U.dtype)], axis=0)
    Lp = np.concatenate([Lam, np.zeros((1, Lam.shape[1]), dtype=Lam.dtype)], axis=0)
    d = np.where(topo.tet_dofs >= 0, topo.tet_dofs, n)
    ut = Up[d]   # [nt, nl, m]
    lt = Lp[d]
    G = (k0 * k0) * np.einsum("tim,tij,tjm->t", lt, M, ut)
    ft, fl = impedance_faces(topo)
    if ft.size:
        B = face_matrix(xyz, topo, ft, fl)
        gb = np.einsum("fim,fij,fjm->f", lt[ft], B, ut[ft])
        coef = -1j * k0 / (2.0 * np.sqrt(eps[ft]))
        np.add.at(G, ft, coef * gb)
    return np.conj(G)


def forward(xyz, topo, eps, freq, tx, rx, A=None):
    """Assemble, solve every transmitter, and return (S, U, A, lu, rx map)."""
    if A is None:
        A = assemble_system(xyz, topo, eps, freq)
    tx = np.asarray(tx, dtype=np.float64).reshape(-1, 8)
    rx = np.asarray(rx, dtype=np.float64).reshape(-1, 8)
    tdof, tsgn = antenna_edges(xyz, topo, tx)
    rdof, rsgn = antenna_edges(xyz, topo, rx)
    b = build_rhs(topo.ndof, tdof, tsgn, tx[:, 6] + 1j * tx[:, 7], freq)
    U, lu = direct_solve(A, b)
    S = s_matrix(U, rdof, rsgn)
    return dict(S=S, U=U, A=A, lu=lu, b=b, rx_dofs=rdof, rx_signs=rsgn, tx_dofs=tdof, tx_signs=tsgn)


def misfit_and_gradient(xyz, topo, eps, freq, tx, rx, S_meas, w=None, fwd=None):
    """J, conj(G) per tet and the adjoint fields, with the state from ``forward``."""
    if fwd is None:
        fwd = forward(xyz, topo, eps, freq, tx, rx)
    J, r = misfit(fwd["S"], S_meas, w)
    g = adjoint_rhs(topo.ndof, r, w, fwd["rx_dofs"], fwd["rx_signs"])
    Lam = fwd["lu"].solve(g)
    grad = gradient(xyz, topo, eps, freq, fwd["U"], Lam)
    return J, grad, dict(fwd, Lam=Lam, g=g, r=r)
