"""Nedelec basis functions and element integrals by numerical quadrature (Section 2.1).

Barycentric coordinates lambda_0..3 of a tet with vertices sorted by global id.
Whitney (degree 1):  N_ab = lambda_a grad(lambda_b) - lambda_b grad(lambda_a),
                     curl N_ab = 2 grad(lambda_a) x grad(lambda_b).
Second order adds    grad(lambda_a lambda_b) = lambda_a grad(lambda_b) + lambda_b grad(lambda_a)
(curl free) and per face (a < b < c) lambda_c N_ab and lambda_a N_bc, with
curl(phi N) = grad(phi) x N + phi curl N.

Integrals use collapsed (Duffy) Gauss-Legendre product rules on the reference
tet and triangle, exact for the polynomial degrees involved.
"""

import numpy as np

from .topology import LOCAL_EDGES, LOCAL_FACES, OPPOSITE


def _gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def tet_rule(n):
    """Points as barycentric coordinates [nq, 4], weights [nq] summing to 1/6.

    Duffy map xi1 = u, xi2 = v (1 - u), xi3 = w (1 - u)(1 - v), Jacobian
    (1 - u)^2 (1 - v); exact for total degree <= 2n - 3.
    """
    x, w = _gl01(n)
    U, V, W = np.meshgrid(x, x, x, indexing="ij")
    WU, WV, WW = np.meshgrid(w, w, w, indexing="ij")
    xi1 = U
    xi2 = V * (1.0 - U)
    xi3 = W * (1.0 - U) * (1.0 - V)
    wt = WU * WV * WW * (1.0 - U) ** 2 * (1.0 - V)
    lam = np.stack([1.0 - xi1 - xi2 - xi3, xi1, xi2, xi3], axis=-1).reshape(-1, 4)
    return lam, wt.ravel()


def tri_rule(n):
    """Points as barycentric coordinates [nq, 3], weights summing to 1/2 (exact to 2n - 2)."""
    x, w = _gl01(n)
    U, V = np.meshgrid(x, x, indexing="ij")
    WU, WV = np.meshgrid(w, w, indexing="ij")
    s1 = U
    s2 = V * (1.0 - U)
    wt = WU * WV * (1.0 - U)
    lam = np.stack([1.0 - s1 - s2, s1, s2], axis=-1).reshape(-1, 3)
    return lam, wt.ravel()


def bary_gradients(P):
    """P: [nt, 4, 3] vertex coordinates.  Returns grad(lambda) [nt, 4, 3] and |det| [nt]."""
    E = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)  # columns
    Einv = np.linalg.inv(E)  # rows are grad(xi_k)
    G = np.empty_like(P)
    G[:, 1:] = Einv
    G[:, 0] = -Einv.sum(axis=1)
    return G, np.abs(np.linalg.det(E))


def basis_at(lam, G, order):
    """Basis values and curls.

    lam: [nq, 4] barycentric points; G: [nt, 4, 3].
    Returns N [nt, nq, nl, 3] and curl N [nt, nq, nl, 3].
    """
    nt = G.shape[0]
    nq = lam.shape[0]
    L = np.broadcast_to(lam[None, :, :, None], (nt, nq, 4, 1))
    Gq = np.broadcast_to(G[:, None, :, :], (nt, nq, 4, 3))

    def whitney(a, b):
        n = L[:, :, a] * Gq[:, :, b] - L[:, :, b] * Gq[:, :, a]
        c = np.broadcast_to(2.0 * np.cross(G[:, a], G[:, b])[:, None, :], (nt, nq, 3))
        return n, c

    vals, curls = [], []
    for a, b in LOCAL_EDGES:
        n, c = whitney(a, b)
        vals.append(n)
        curls.append(c)
    if order == 2:
        zero = np.zeros((nt, nq, 3))
        for a, b in LOCAL_EDGES:
            vals.append(L[:, :, a] * Gq[:, :, b] + L[:, :, b] * Gq[:, :, a])
            curls.append(zero)
        for a, b, c in LOCAL_FACES:
            for (p, q), r in (((a, b), c), ((b, c), a)):
                n, cn = whitney(p, q)
                vals.append(L[:, :, r] * n)
                curls.append(np.cross(Gq[:, :, r], n) + L[:, :, r] * cn)
    return np.stack(vals, axis=2), np.stack(curls, axis=2)


def _rule_n(order):
    return 3 if order == 1 else 4


def element_matrices(xyz, topo, tets=None, chunk=8192):
    """K_t = int curl N_i . curl N_j and M_t = int N_i . N_j, [nt, nl, nl] float64.

    Both are symmetrised exactly, (X + X^T) / 2, so that the assembled matrix
    is complex symmetric bit for bit (the form of Eq. pbdirectvarf is bilinear).
    """
    tv = topo.tv if tets is None else topo.tv[tets]
    lam, w = tet_rule(_rule_n(topo.order))
    nt = tv.shape[0]
    nl = topo.nl
    K = np.empty((nt, nl, nl))
    M = np.empty((nt, nl, nl))
    for s in range(0, nt, chunk):
        P = xyz[tv[s:s + chunk]]
        G, det = bary_gradients(P)
        N, C = basis_at(lam, G, topo.order)
        k = np.einsum("q,tqia,tqja->tij", w, C, C) * det[:, None, None]
        m = np.einsum("q,tqia,tqja->tij", w, N, N) * det[:, None, None]
        K[s:s + chunk] = 0.5 * (k + k.transpose(0, 2, 1))
        M[s:s + chunk] = 0.5 * (m + m.transpose(0, 2, 1))
    return K, M


def face_matrix(xyz, topo, tets, lfaces):
    """B_f = int_f (N_i x n) . (N_j x n) over local face lfaces[k] of tet tets[k].

    Returns [nf, nl, nl] in the owning tet's local numbering (DOFs not on the
    face give zero rows).  Tangential part N_T = N - (N . n) n, n = unit normal.
    """
    tets = np.asarray(tets, dtype=np.int64)
    lfaces = np.asarray(lfaces, dtype=np.int64)
    nf = tets.shape[0]
    nl = topo.nl
    out = np.zeros((nf, nl, nl))
    if nf == 0:
        return out
    lam3, w = tri_rule(3 if topo.order == 1 else 4)
    P = xyz[topo.tv[tets]]
    G, _ = bary_gradients(P)
    for f in range(4):
        sel = np.nonzero(lfaces == f)[0]
        if sel.size == 0:
            continue
        fverts = LOCAL_FACES[f]
        lam = np.zeros((lam3.shape[0], 4))
        lam[:, fverts] = lam3
        Gs = G[sel]
        N, _ = basis_at(lam, Gs, topo.order)
        nrm = Gs[:, OPPOSITE[f]]
        nrm = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
        NT = N - np.einsum("tqia,ta->tqi", N, nrm)[..., None] * nrm[:, None, None, :]
        Pf = P[sel][:, fverts]
        area2 = np.linalg.norm(np.cross(Pf[:, 1] - Pf[:, 0], Pf[:, 2] - Pf[:, 0]), axis=1)
        b = np.einsum("q,tqia,tqja->tij", w, NT, NT) * area2[:, None, None]
        out[sel] = 0.5 * (b + b.transpose(0, 2, 1))
    return out
