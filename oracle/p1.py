"""Nodal (P1) permittivity parameter, Tikhonov regularisation and normalised
misfit weights -- oracle, test infrastructure only.

The inversion of the paper uses a P1 parameter (Section 6.3) and a normalised
misfit with a gradient penalty (Eq. defJ2).  With a per-vertex relative
permittivity kappa_v:

* each tet's permittivity is the P1 field at its centroid, eps_t = (1/4) sum of
  kappa at its four vertices (the tet-centroid sampling used for every map);
* the penalty is R = (alpha / 2) * integral of |grad kappa|^2 over the mesh =
  (alpha / 2) Re(kappa^H K kappa) with K the P1 stiffness matrix (real,
  symmetric, element matrices |t| grad(lambda_a) . grad(lambda_b));
* the gradient of J(eps(kappa)) + R(kappa) in the convention of the per-tet
  gradient (dPhi/dRe + i dPhi/dIm) is the per-tet gradient spread back to the
  vertices with weight 1/4 plus alpha K kappa;
* the normalised weights are w_ij = 1 / |S^empty_ij|^2, S^empty being the
  S-matrix of the empty (gel-filled) chamber.

Parity status: pinned by tests/test_oracle_p1.py (K annihilates constants, the
energy of a linear field equals |grad|^2 times the volume, K symmetric positive
semidefinite, the spreading is the adjoint of the centroid sampling, and central
finite differences of the full objective).
"""

import numpy as np
import scipy.sparse as sp

from .fem import bary_gradients
from .solve import forward, misfit_and_gradient


def p1_to_tet(tet, kappa):
    """eps_t = mean of kappa over the tet's four vertices."""
    return kappa[tet].mean(axis=1)


def p1_spread(tet, nv, grad_tet):
    """Adjoint of p1_to_tet for the real inner product: g_v = 1/4 sum_{t contains v} g_t."""
    g = np.zeros(nv, dtype=complex)
    for a in range(4):
        np.add.at(g, tet[:, a], 0.25 * grad_tet)
    return g


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


def objective_p1(xyz, topo, tet, kappa, freq, tx, rx, S_meas, w, alpha, K):
    """Phi = J(eps(kappa)) + R(kappa) and its per-vertex gradient."""
    eps = p1_to_tet(tet, kappa)
    J, grad_t, _ = misfit_and_gradient(xyz, topo, eps, freq, tx, rx, S_meas, w)
    R, gR = regularisation(K, kappa, alpha)
    return J + R, p1_spread(tet, xyz.shape[0], grad_t) + gR


def empty_chamber_weights(xyz, topo, eps_empty, freq, tx, rx):
    """Normalised misfit weights from the S-matrix of the empty chamber."""
    return normalised_weights(forward(xyz, topo, eps_empty, freq, tx, rx)["S"])
