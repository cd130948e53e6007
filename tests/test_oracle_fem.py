"""Pins for the oracle's element integrals (Section 2.1).

The oracle integrates by quadrature with basis values built by the product
rule.  Here the same integrals are computed a second, independent way: each
basis function is expanded into barycentric monomials times constant vectors,
curls are taken monomial by monomial (curl(lambda^a v) = sum_k a_k
lambda^(a - e_k) grad(lambda_k) x v), and every monomial is integrated with
the closed form  int_t lambda^a = 6 |t| a! / (|a| + 3)!  (faces:
2 |f| a! / (|a| + 2)!).
"""

import itertools
from math import factorial

import numpy as np
import pytest

import oracle as O
from oracle.fem import bary_gradients, tet_rule, tri_rule
from oracle.topology import LOCAL_EDGES, LOCAL_FACES, OPPOSITE

pytestmark = pytest.mark.filterwarnings("ignore")


def _mono_int_tet(alpha, vol):
    s = sum(alpha)
    return 6.0 * vol * np.prod([factorial(a) for a in alpha]) / factorial(s + 3)


def _mono_int_face(alpha, area):
    s = sum(alpha)
    return 2.0 * area * np.prod([factorial(a) for a in alpha]) / factorial(s + 2)


def _e(k):
    v = [0, 0, 0, 0]
    v[k] = 1
    return tuple(v)


def _add(a, b):
    return tuple(x + y for x, y in zip(a, b))


def _poly_basis(G, order):
    """List of vector polynomials {alpha: vec} in the oracle's local order."""
    def whitney(a, b):
        return {_e(a): G[b].copy(), _e(b): -G[a].copy()}

    out = [whitney(a, b) for a, b in LOCAL_EDGES]
    if order == 2:
        for a, b in LOCAL_EDGES:
            out.append({_e(a): G[b].copy(), _e(b): G[a].copy()})
        for a, b, c in LOCAL_FACES:
            for (p, q), r in (((a, b), c), ((b, c), a)):
                w = whitney(p, q)
                out.append({_add(k, _e(r)): v for k, v in w.items()})
    return out


def _poly_curl(P, G):
    out = {}
    for alpha, v in P.items():
        for k in range(4):
            if alpha[k] == 0:
                continue
            beta = list(alpha)
            beta[k] -= 1
            beta = tuple(beta)
            out[beta] = out.get(beta, np.zeros(3)) + alpha[k] * np.cross(G[k], v)
    return out


def _poly_dot_int(P, Q, vol):
    s = 0.0
    for a, u in P.items():
        for b, v in Q.items():
            s += float(u @ v) * _mono_int_tet(_add(a, b), vol)
    return s


def _poly_face_int(P, Q, n, area, d):
    s = 0.0
    for a, u in P.items():
        for b, v in Q.items():
            g = _add(a, b)
            if g[d] != 0:
                continue  # lambda_d = 0 on the face opposite vertex d
            s += (float(u @ v) - float(u @ n) * float(v @ n)) * _mono_int_face(g, area)
    return s


def _random_tet(seed):
    rng = np.random.default_rng(seed)
    while True:
        P = rng.uniform(-1.0, 1.0, size=(4, 3))
        vol = abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], 1))) / 6.0
        if vol > 0.05:
            return P


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_element_matrices_match_monomial_closed_form(order, seed):
    P = _random_tet(seed)
    topo = O.build_topology(np.array([[0, 1, 2, 3]]), np.zeros((1, 4), np.int32), 4, order)
    K, M = O.element_matrices(P, topo)
    G, det = bary_gradients(P[None])
    G = G[0]
    vol = det[0] / 6.0
    basis = _poly_basis(G, order)
    curls = [_poly_curl(b, G) for b in basis]
    nl = len(basis)
    Kc = np.array([[_poly_dot_int(curls[i], curls[j], vol) for j in range(nl)] for i in range(nl)])
    Mc = np.array([[_poly_dot_int(basis[i], basis[j], vol) for j in range(nl)] for i in range(nl)])
    assert np.abs(K[0] - Kc).max() <= 1e-12 * np.abs(Kc).max()
    assert np.abs(M[0] - Mc).max() <= 1e-12 * np.abs(Mc).max()


def test_whitney_closed_forms():
    """Order 1 by the textbook closed forms: int lambda_i lambda_j = |t|(1 + d_ij)/20,
    curl N_ab = 2 grad(lambda_a) x grad(lambda_b)."""
    P = _random_tet(5)
    topo = O.build_topology(np.array([[0, 1, 2, 3]]), np.zeros((1, 4), np.int32), 4, 1)
    K, M = O.element_matrices(P, topo)
    G, det = bary_gradients(P[None])
    G = G[0]
    vol = det[0] / 6.0

    def mm(i, j):
        return vol * (1.0 + (i == j)) / 20.0

    for e, (a, b) in enumerate(LOCAL_EDGES):
        for f, (c, d) in enumerate(LOCAL_EDGES):
            m = (mm(a, c) * G[b] @ G[d] - mm(a, d) * G[b] @ G[c]
                 - mm(b, c) * G[a] @ G[d] + mm(b, d) * G[a] @ G[c])
            k = 4.0 * vol * np.cross(G[a], G[b]) @ np.cross(G[c], G[d])
            assert abs(M[0, e, f] - m) <= 1e-13 * abs(M[0]).max()
            assert abs(K[0, e, f] - k) <= 1e-13 * abs(K[0]).max()


@pytest.mark.parametrize("order", [1, 2])
def test_face_matrix_matches_closed_form(order):
    P = _random_tet(7)
    topo = O.build_topology(np.array([[0, 1, 2, 3]]), np.zeros((1, 4), np.int32), 4, order)
    G, _ = bary_gradients(P[None])
    G = G[0]
    basis = _poly_basis(G, order)
    for f in range(4):
        B = O.face_matrix(P, topo, [0], [f])[0]
        d = OPPOSITE[f]
        n = G[d] / np.linalg.norm(G[d])
        a, b, c = LOCAL_FACES[f]
        area = 0.5 * np.linalg.norm(np.cross(P[b] - P[a], P[c] - P[a]))
        nl = len(basis)
        Bc = np.array([[_poly_face_int(basis[i], basis[j], n, area, d) for j in range(nl)]
                       for i in range(nl)])
        assert np.abs(B - Bc).max() <= 1e-12 * np.abs(Bc).max()


@pytest.mark.parametrize("n,deg", [(3, 3), (4, 5), (5, 7)])
def test_tet_rule_exact_for_monomials(n, deg):
    lam, w = tet_rule(n)
    assert abs(w.sum() - 1.0 / 6.0) < 1e-15
    for alpha in itertools.product(range(deg + 1), repeat=4):
        if sum(alpha) > deg:
            continue
        q = np.sum(w * np.prod(lam ** np.array(alpha), axis=1))
        assert abs(q - _mono_int_tet(alpha, 1.0 / 6.0)) < 1e-15


@pytest.mark.parametrize("n,deg", [(3, 4), (4, 6)])
def test_tri_rule_exact_for_monomials(n, deg):
    lam, w = tri_rule(n)
    for alpha in itertools.product(range(deg + 1), repeat=3):
        if sum(alpha) > deg:
            continue
        q = np.sum(w * np.prod(lam ** np.array(alpha), axis=1))
        assert abs(q - _mono_int_face(alpha, 0.5)) < 1e-15


def test_order2_space_dimension_and_whitney_complex():
    """The 20 order-2 functions are linearly independent and the first 12 span P1^3."""
    P = _random_tet(9)
    G, _ = bary_gradients(P[None])
    lam, _ = tet_rule(4)
    N, _ = O.basis_at(lam, G, 2)
    mat = N[0].transpose(1, 0, 2).reshape(20, -1)
    assert np.linalg.matrix_rank(mat, tol=1e-10) == 20
    # constant and linear fields x_k e_l belong to span of the first 12 (full P1^3)
    pts = P[None, None, :, :]
    xq = np.einsum("qk,kd->qd", lam, P)
    targets = []
    for l in range(3):
        e = np.zeros(3)
        e[l] = 1.0
        targets.append(np.broadcast_to(e, xq.shape))
        for k in range(3):
            targets.append(xq[:, k:k + 1] * e[None, :])
    B12 = mat[:12]
    for t in targets:
        coef, res, *_ = np.linalg.lstsq(B12.T, t.ravel(), rcond=None)
        assert np.linalg.norm(B12.T @ coef - t.ravel()) < 1e-10 * max(1.0, np.linalg.norm(t))
