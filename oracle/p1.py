"""Nodal (P1) permittivity parameter, Tikhonov regularisation and normalised
misfit weights -- oracle, test infrastructure only.

The inversion of the paper uses a piecewise-linear parameter on the state mesh
(Section 6.3) and the normalised, regularised misfit of Eq. defJ2.  With a
per-vertex relative permittivity kappa_v (the paper's kappa = k0^2 eps_r; the
factor k0^2 stays in the operator so that kappa and eps_r share units), the
P1 field is kappa(x) = sum_v kappa_v lambda_v(x) and the mass term of the
variational form (Eq. pbdirectvarf) becomes

    int_t kappa N_i . N_j = sum_{w=0..3} kappa_{v_w(t)} M_t^(w)[i, j],
    M_t^(w)[i, j] = int_t lambda_w N_i . N_j          (vertex-weighted masses),

so A(kappa) = K - k0^2 sum_t sum_w kappa_{v_w(t)} M_t^(w) + i sum_f beta_f B_f.
The M_t^(w) are integrated by the same collapsed Gauss-Legendre rule as the
element matrices (degree 3 for order 1, 5 for order 2: exact).

Reading (the paper does not say how beta and the interface wavenumber of the
ORAS local problems follow a P1 kappa): both take the P1 field at the owning
tet's centroid, kappa_bar_t = (1/4) sum_w kappa_{v_w(t)}, i.e.
beta_f = k0 sqrt(kappa_bar_t) for the tet t owning face f.

Gradient (Section 5 in discrete form, derived like the per-tet gradient of
``solve``): with r = S - S_meas, g_j = sum_i w_ij r_ij q_i and
lambda_j = A^{-1} g_j,

    G_v = sum_{(t, w): v_w(t) = v} [ k0^2 sum_j lambda_{j,t}^T M_t^(w) u_{j,t}
                                     + (1/4) sum_j lambda_{j,t}^T (-i k0 / (2 sqrt(kappa_bar_t))) B_t u_{j,t} ],
    dJ/dRe(kappa_v) + i dJ/dIm(kappa_v) = conj(G_v),

B_t summing the face matrices of the impedance faces owned by t.

Penalty (Eq. defJ2): R = (alpha / 2) int |grad kappa|^2 = (alpha / 2)
Re(kappa^H K kappa), K the P1 stiffness matrix; its gradient is alpha K kappa.
Normalised weights: w_ij = 1 / |S^empty_ij|^2 (Eq. defJ2), S^empty the
S-matrix of the empty (gel-filled) chamber.

Parity status: pinned by tests/test_oracle_p1.py -- the four vertex masses sum
to the element mass of ``fem`` (itself pinned by closed forms), an independent
monomial closed form of every M_t^(w) for Whitney elements, a constant kappa
reproducing the P0 operator of ``assemble``, the stiffness identities (constants
annihilated, |a|^2 times the volume for a linear field, positive
semidefinite), and central finite differences of the full objective in Re and
Im of kappa at sampled vertices, impedance-face vertices included.
"""

import numpy as np
import scipy.sparse as sp

from .assemble import _scatter_symmetric, impedance_faces
from .constants import k0_of
from .fem import _rule_n, bary_gradients, basis_at, element_matrices, face_matrix, tet_rule
from .solve import adjoint_rhs, direct_solve, misfit, s_matrix
from .assemble import antenna_edges, build_rhs


def vertex_mass_matrices(xyz, topo, chunk=4096):
    """M_t^(w)[i, j] = int_t lambda_w N_i . N_j, [nt, 4, nl, nl] float64, w in
    the tet's sorted local vertex order (topo.tv).  Symmetrised exactly."""
    lam, wq = tet_rule(_rule_n(topo.order))
    tv = topo.tv
    nt, nl = tv.shape[0], topo.nl
    out = np.empty((nt, 4, nl, nl))
    for s in range(0, nt, chunk):
        G, det = bary_gradients(xyz[tv[s:s + chunk]])
        N, _ = basis_at(lam, G, topo.order)
        m = np.einsum("q,qw,tqia,tqja->twij", wq, lam, N, N) * det[:, None, None, None]
        out[s:s + chunk] = 0.5 * (m + m.transpose(0, 1, 3, 2))
    return out


def centroid_values(topo, kappa):
    """kappa_bar_t = (1/4) sum of kappa over the tet's vertices (the P1 field at its centroid)."""
    return np.asarray(kappa, dtype=np.complex128)[topo.tv].mean(axis=1)


def assemble_system_p1(xyz, topo, kappa, freq, K=None, Mv=None):
    """A(kappa) of the module docstring (complex symmetric CSR)."""
    kappa = np.asarray(kappa, dtype=np.complex128)
    k0 = k0_of(freq)
    if K is None:
        K, _ = element_matrices(xyz, topo)
    if Mv is None:
        Mv = vertex_mass_matrices(xyz, topo)
    kw = kappa[topo.tv]                                   # [nt, 4]
    vol = K.astype(np.complex128) - (k0 * k0) * np.einsum("tw,twij->tij", kw, Mv)
    ft, fl = impedance_faces(topo)
    B = face_matrix(xyz, topo, ft, fl)
    beta = k0 * np.sqrt(centroid_values(topo, kappa)[ft])
    bnd = 1j * beta[:, None, None] * B
    dofs = np.concatenate([topo.tet_dofs, topo.tet_dofs[ft]], axis=0)
    vals = np.concatenate([vol, bnd], axis=0)
    return _scatter_symmetric(dofs, vals, topo.ndof)


def forward_p1(xyz, topo, kappa, freq, tx, rx, Mv=None):
    """Assemble A(kappa), solve every transmitter, S-parameters (Eq. sij)."""
    A = assemble_system_p1(xyz, topo, kappa, freq, Mv=Mv)
    tx = np.asarray(tx, dtype=np.float64).reshape(-1, 8)
    rx = np.asarray(rx, dtype=np.float64).reshape(-1, 8)
    tdof, tsgn = antenna_edges(xyz, topo, tx)
    rdof, rsgn = antenna_edges(xyz, topo, rx)
    b = build_rhs(topo.ndof, tdof, tsgn, tx[:, 6] + 1j * tx[:, 7], freq)
    U, lu = direct_solve(A, b)
    return dict(S=s_matrix(U, rdof, rsgn), U=U, A=A, lu=lu, rx_dofs=rdof, rx_signs=rsgn)


def gradient_p1(xyz, topo, kappa, freq, U, Lam, Mv=None):
    """conj(G_v) for every vertex (module docstring)."""
    k0 = k0_of(freq)
    if Mv is None:
        Mv = vertex_mass_matrices(xyz, topo)
    n = topo.ndof
    Up = np.concatenate([U, np.zeros((1, U.shape[1]), dtype=U.dtype)], axis=0)
    Lp = np.concatenate([Lam, np.zeros((1, Lam.shape[1]), dtype=Lam.dtype)], axis=0)
    d = np.where(topo.tet_dofs >= 0, topo.tet_dofs, n)
    ut, lt = Up[d], Lp[d]                                  # [nt, nl, m]
    Gtw = (k0 * k0) * np.einsum("tim,twij,tjm->tw", lt, Mv, ut)
    ft, fl = impedance_faces(topo)
    if ft.size:
        B = face_matrix(xyz, topo, ft, fl)
        gb = np.einsum("fim,fij,fjm->f", lt[ft], B, ut[ft])
        coef = -1j * k0 / (2.0 * np.sqrt(centroid_values(topo, kappa)[ft]))
        for w in range(4):
            np.add.at(Gtw[:, w], ft, 0.25 * coef * gb)
    nv = xyz.shape[0]
    G = np.zeros(nv, dtype=np.complex128)
    for w in range(4):
        np.add.at(G, topo.tv[:, w], Gtw[:, w])
    return np.conj(G)


def p1_stiffness(xyz, tet):
    """P1 stiffness matrix K (real CSR, nv x nv): K_e[a][b] = |t| grad(lambda_a) . grad(lambda_b)."""
    G, det = bary_gradients(xyz[tet])
    vol = det / 6.0
    Ke = np.einsum("tai,tbi->tab", G, G) * vol[:, None, None]
    rows = np.repeat(tet, 4, axis=1).ravel()
    cols = np.tile(tet, (1, 4)).ravel()
    nv = xyz.shape[0]
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(nv, nv)).tocsr()


def regularisation(K, kappa, alpha):
    """R = (alpha/2) Re(kappa^H K kappa) and its gradient alpha K kappa (dR/dRe + i dR/dIm)."""
    Kk = K @ kappa
    return 0.5 * alpha * float(np.real(np.vdot(kappa, Kk))), alpha * Kk


def normalised_weights(S_empty):
    """w_ij = 1 / |S^empty_ij|^2."""
    return 1.0 / np.abs(S_empty) ** 2


def objective_p1(xyz, topo, kappa, freq, tx, rx, S_meas, w, alpha, K, Mv=None):
    """Phi = J(kappa) + R(kappa) (Eq. defJ2 with the weights w) and its
    per-vertex gradient dPhi/dRe + i dPhi/dIm; also returns J and R."""
    if Mv is None:
        Mv = vertex_mass_matrices(xyz, topo)
    fwd = forward_p1(xyz, topo, kappa, freq, tx, rx, Mv=Mv)
    J, r = misfit(fwd["S"], S_meas, w)
    g = adjoint_rhs(topo.ndof, r, w, fwd["rx_dofs"], fwd["rx_signs"])
    Lam = fwd["lu"].solve(g)
    grad = gradient_p1(xyz, topo, kappa, freq, fwd["U"], Lam, Mv=Mv)
    R, gR = regularisation(K, kappa, alpha)
    return J + R, grad + gR, dict(J=J, R=R, S=fwd["S"], U=fwd["U"], Lam=Lam)


def empty_chamber_weights(xyz, topo, eps_empty, freq, tx, rx):
    """Normalised misfit weights from the S-matrix of the empty (gel-filled) chamber."""
    from .solve import forward
    return normalised_weights(forward(xyz, topo, eps_empty, freq, tx, rx)["S"])
