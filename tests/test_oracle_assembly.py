"""Pins for the oracle's global assembly (Section 2, Eq. pbdirectvarf and Eq. linsys).

* discrete de Rham: curl-curl applied to gradients is zero (K G = 0);
* the bilinear form gives an exactly complex-symmetric A;
* a plane-wave manufactured solution E = p exp(-i k d.x) of the impedance
  problem converges at rate 1 (order 1) and 2 (order 2) in L2;
* the +i beta sign is the outgoing condition for the exp(+i w t) convention:
  on the face the plane wave leaves through, its boundary datum vanishes.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
from oracle.assemble import _scatter_symmetric
from oracle.fem import bary_gradients, basis_at, tet_rule, tri_rule
from oracle.topology import LOCAL_FACES, OPPOSITE
from synthetic import chamber_mesh, cube_mesh


def _curlcurl(mesh, order):
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    K, _ = O.element_matrices(mesh.xyz, topo)
    return topo, _scatter_symmetric(topo.tet_dofs, K, topo.ndof)


@pytest.mark.parametrize("order", [1, 2])
def test_curl_grad_is_zero_cube(order):
    mesh = cube_mesh(4, jitter=0.0)
    topo, K = _curlcurl(mesh, order)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(mesh.nv)
    x = np.zeros(topo.ndof)
    w = topo.dof_kind == 0
    v = topo.dof_verts
    x[w] = phi[v[w, 1]] - phi[v[w, 0]]  # Whitney DOFs of grad(P1): phi(high) - phi(low)
    if order == 2:
        g = topo.dof_kind == 1
        x[g] = rng.standard_normal(g.sum())  # gradients of edge bubbles
    y = K @ x
    assert np.linalg.norm(y) <= 1e-13 * abs(K).max() * np.linalg.norm(x)


def test_curl_grad_is_zero_chamber_with_pec():
    mesh = chamber_mesh(8, 8)
    topo, K = _curlcurl(mesh, 1)
    rng = np.random.default_rng(1)
    phi = rng.standard_normal(mesh.nv)
    pec_v = np.zeros(mesh.nv, dtype=bool)
    pec_v[topo.edges[topo.pec_edge].ravel()] = True
    phi[pec_v] = 0.0  # gradient fields with zero tangential trace on the PEC wall
    v = topo.dof_verts
    x = phi[v[:, 1]] - phi[v[:, 0]]
    assert np.linalg.norm(K @ x) <= 1e-13 * abs(K).max() * np.linalg.norm(x)
    assert np.linalg.norm(x) > 0


@pytest.mark.parametrize("order", [1, 2])
def test_A_exactly_symmetric(order):
    mesh = chamber_mesh(8, 8)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    eps = np.full(mesh.nt, 44 - 20j)
    A = O.assemble_system(mesh.xyz, topo, eps, 1e9)
    assert (A - A.T).count_nonzero() == 0 or abs(A - A.T).max() == 0.0


def test_matrix_sizes_match_grid_counts():
    """Kuhn cube 8^3: 729 vertices, 3072 tets; edges = 7 n^3 + 3 n^2 ... counted directly."""
    mesh = cube_mesh(8)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    n = 8
    # edges of a Kuhn-split grid: axis edges 3 n (n+1)^2, face diagonals 3 n^2 (n+1), body diagonals n^3
    assert topo.edges.shape[0] == 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3
    assert topo.ndof == 4184


# --- plane wave -------------------------------------------------------------

FREQ = 1e9
EPS_PW = 4.0 - 1.0j
D = np.array([1.0, 2.0, 2.0]) / 3.0
Pv = np.array([2.0, -1.0, 0.0]) / np.sqrt(5.0)


def _plane_wave(x, k):
    ph = np.exp(-1j * k * (x @ D))
    E = ph[..., None] * Pv
    curlE = (-1j * k) * ph[..., None] * np.cross(D, Pv)
    return E, curlE


def _manufactured_error(n, order):
    mesh = cube_mesh(n, jitter=0.0, permute=True)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    k0 = O.k0_of(FREQ)
    k = k0 * np.sqrt(EPS_PW)
    eps = np.full(mesh.nt, EPS_PW)
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ)
    # boundary datum g = (curl E) x n + i beta n x (E x n), beta = k, n outward
    f = np.nonzero(topo.face_tag == 2)[0]
    ft, fl = topo.face_tets[f, 0], topo.face_local[f, 0]
    lam3, w3 = tri_rule(7)
    F = np.zeros(topo.ndof, dtype=np.complex128)
    P = mesh.xyz[topo.tv[ft]]
    G, _ = bary_gradients(P)
    for lf in range(4):
        sel = np.nonzero(fl == lf)[0]
        if sel.size == 0:
            continue
        lam = np.zeros((lam3.shape[0], 4))
        lam[:, LOCAL_FACES[lf]] = lam3
        N, _ = basis_at(lam, G[sel], order)
        nout = -G[sel, OPPOSITE[lf]]
        nout /= np.linalg.norm(nout, axis=1, keepdims=True)
        xq = np.einsum("qk,tkd->tqd", lam, P[sel])
        E, cE = _plane_wave(xq, k)
        En = np.einsum("tqd,td->tq", E, nout)
        ET = E - En[..., None] * nout[:, None, :]
        g = np.cross(cE, nout[:, None, :]) + 1j * k * ET
        Pf = P[sel][:, LOCAL_FACES[lf]]
        area2 = np.linalg.norm(np.cross(Pf[:, 1] - Pf[:, 0], Pf[:, 2] - Pf[:, 0]), axis=1)
        loc = np.einsum("q,tqd,tqid->ti", w3, g, N) * area2[:, None]
        d = topo.tet_dofs[ft[sel]]
        np.add.at(F, d.ravel(), loc.ravel())
    u = spla.spsolve(A.tocsc(), F)
    # L2 error by quadrature
    lam, w = tet_rule(5)
    up = u[topo.tet_dofs]
    err2 = 0.0
    ref2 = 0.0
    for s in range(0, mesh.nt, 4096):
        P = mesh.xyz[topo.tv[s:s + 4096]]
        G, det = bary_gradients(P)
        N, _ = basis_at(lam, G, order)
        Eh = np.einsum("ti,tqid->tqd", up[s:s + 4096], N)
        xq = np.einsum("qk,tkd->tqd", lam, P)
        E, _ = _plane_wave(xq, k)
        err2 += np.sum(w[None, :, None] * det[:, None, None] * np.abs(Eh - E) ** 2)
        ref2 += np.sum(w[None, :, None] * det[:, None, None] * np.abs(E) ** 2)
    return np.sqrt(err2 / ref2)


def test_plane_wave_outgoing_datum_vanishes():
    k = O.k0_of(FREQ) * np.sqrt(EPS_PW)
    x = np.random.default_rng(3).uniform(0, 0.1, size=(20, 3))
    E, cE = _plane_wave(x, k)
    n = D  # exit face normal equal to the propagation direction
    ET = E - (E @ n)[:, None] * n
    g = np.cross(cE, n) + 1j * k * ET
    assert np.abs(g).max() < 1e-12 * np.abs(cE).max()


def test_plane_wave_convergence_order1():
    errs = [_manufactured_error(n, 1) for n in (4, 8, 16)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.1
    assert np.all(rates > 0.85) and np.all(rates < 1.3), (errs, rates)


@pytest.mark.slow
def test_plane_wave_convergence_order2():
    errs = [_manufactured_error(n, 2) for n in (2, 4, 8)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 0.02
    assert rates[-1] > 1.8 and rates[-1] < 2.4, (errs, rates)
