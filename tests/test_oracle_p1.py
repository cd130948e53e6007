"""Pins for the oracle's nodal (P1) parameter: the vertex-weighted mass term,
the gradient penalty and the normalised weights (Eq. defJ2, the P1 parameter
of Section 6.3).

* the four vertex masses of a tet sum to its element mass (sum_w lambda_w = 1),
  the element mass being pinned in test_oracle_fem.py by closed forms;
* every Whitney vertex mass equals an independent monomial closed form,
  int_t lambda^a = 6 |t| a! / (|a| + 3)!, on random tets;
* a constant kappa gives the P0 operator of ``assemble`` with eps_r = kappa;
* the P1 stiffness matrix annihilates constants, is symmetric positive
  semidefinite, and gives |a|^2 times the volume for a linear field a.x + b;
* the gradient of the full objective (normalised misfit + penalty) equals
  central finite differences in Re and Im of kappa at sampled vertices,
  vertices of impedance faces included (they carry the beta term).
"""

from math import factorial

import numpy as np
import pytest

import oracle as O
from oracle import p1
from synthetic import antenna_array, chamber_mesh, cube_antennas, cube_mesh

FREQ = 1e9


def _moment(alpha, vol):
    s = sum(alpha)
    return 6.0 * vol * np.prod([factorial(a) for a in alpha]) / factorial(s + 3)


@pytest.mark.parametrize("order", [1, 2])
def test_vertex_masses_sum_to_element_mass(order):
    mesh = cube_mesh(2)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    _, M = O.element_matrices(mesh.xyz, topo)
    Mv = p1.vertex_mass_matrices(mesh.xyz, topo)
    assert np.abs(Mv.sum(axis=1) - M).max() <= 1e-14 * np.abs(M).max()
    # each vertex mass is symmetric and not a quarter of M (kappa varies inside the tet)
    assert np.abs(Mv - Mv.transpose(0, 1, 3, 2)).max() == 0.0
    assert np.abs(Mv[:, 0] - 0.25 * M).max() > 1e-3 * np.abs(M).max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_whitney_vertex_mass_closed_form(seed):
    rng = np.random.default_rng(seed)
    xyz = rng.standard_normal((4, 3))
    tet = np.array([[0, 1, 2, 3]])
    tag = np.zeros((1, 4), dtype=np.int32)
    topo = O.build_topology(tet, tag, 4, 1)
    Mv = p1.vertex_mass_matrices(xyz, topo)[0]
    G, det = O.fem.bary_gradients(xyz[topo.tv])
    G, vol = G[0], det[0] / 6.0
    edges = O.topology.LOCAL_EDGES
    for w in range(4):
        for i, (a, b) in enumerate(edges):
            for j, (c, d) in enumerate(edges):
                # N_ab . N_cd = sum of +- lambda_x lambda_y grad_u . grad_v
                val = 0.0
                for (x, u, sx) in ((a, b, 1.0), (b, a, -1.0)):
                    for (y, v, sy) in ((c, d, 1.0), (d, c, -1.0)):
                        alpha = [0, 0, 0, 0]
                        alpha[w] += 1
                        alpha[x] += 1
                        alpha[y] += 1
                        val += sx * sy * _moment(alpha, vol) * float(G[u] @ G[v])
                assert abs(Mv[w, i, j] - val) <= 1e-13 * np.abs(Mv).max(), (w, i, j)


@pytest.mark.parametrize("order", [1, 2])
def test_constant_kappa_reproduces_p0_operator(order):
    mesh = cube_mesh(3)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    c = 44.0 - 20.0j
    A1 = p1.assemble_system_p1(mesh.xyz, topo, np.full(mesh.nv, c), FREQ)
    A0 = O.assemble_system(mesh.xyz, topo, np.full(mesh.nt, c), FREQ)
    assert abs(A1 - A0).max() <= 1e-13 * abs(A0).max()
    # and a linear kappa does not
    kap = c + mesh.xyz[:, 0] * 10.0
    A2 = p1.assemble_system_p1(mesh.xyz, topo, kap, FREQ)
    A3 = O.assemble_system(mesh.xyz, topo, p1.centroid_values(topo, kap), FREQ)
    assert abs(A2 - A3).max() > 1e-6 * abs(A3).max()


def test_stiffness_constants_symmetry_and_linear_energy():
    mesh = chamber_mesh(8, 8)
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    nv = mesh.nv
    assert np.abs(K @ np.ones(nv)).max() <= 1e-13 * np.abs(K).max()
    assert abs(K - K.T).max() <= 1e-15 * np.abs(K).max()
    G, det = O.fem.bary_gradients(mesh.xyz[mesh.tet])
    vol = float(np.sum(det) / 6.0)
    rng = np.random.default_rng(1)
    a = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    kap = mesh.xyz @ a + (2.0 - 1.0j)
    energy = float(np.real(np.vdot(kap, K @ kap)))
    assert abs(energy - np.sum(np.abs(a) ** 2) * vol) <= 1e-12 * energy
    small = p1.p1_stiffness(*(lambda m: (m.xyz, m.tet))(cube_mesh(2))).toarray()
    assert np.linalg.eigvalsh(small).min() >= -1e-14 * np.abs(small).max()


def test_objective_gradient_matches_finite_differences():
    mesh = cube_mesh(4)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    tx = antenna_array(cube_antennas())
    rng = np.random.default_rng(3)
    kap_true = 44 - 20j + rng.uniform(-6, 6, mesh.nv) + 1j * rng.uniform(-3, 3, mesh.nv)
    w = p1.empty_chamber_weights(mesh.xyz, topo, np.full(mesh.nt, 44 - 20j), FREQ, tx, tx)
    Mv = p1.vertex_mass_matrices(mesh.xyz, topo)
    S_meas = p1.forward_p1(mesh.xyz, topo, kap_true, FREQ, tx, tx, Mv=Mv)["S"]
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    alpha = 1e-3
    kap = np.full(mesh.nv, 44 - 20j) + rng.uniform(-1, 1, mesh.nv) + 1j * rng.uniform(-1, 1, mesh.nv)
    phi, grad, _ = p1.objective_p1(mesh.xyz, topo, kap, FREQ, tx, tx, S_meas, w, alpha, K, Mv=Mv)
    assert phi > 0
    # two interior vertices and two on the (impedance) boundary of the cube
    on_bnd = np.any((mesh.xyz <= 1e-12) | (mesh.xyz >= 0.1 - 1e-12), axis=1)
    picks = list(rng.choice(np.nonzero(~on_bnd)[0], 2, replace=False)) + \
        list(rng.choice(np.nonzero(on_bnd)[0], 2, replace=False))
    for v in picks:
        for direction, comp in ((1.0, grad[v].real), (1j, grad[v].imag)):
            h = 1e-5 * abs(kap[v])
            kp = kap.copy(); kp[v] += direction * h
            km = kap.copy(); km[v] -= direction * h
            fp = p1.objective_p1(mesh.xyz, topo, kp, FREQ, tx, tx, S_meas, w, alpha, K, Mv=Mv)[0]
            fm = p1.objective_p1(mesh.xyz, topo, km, FREQ, tx, tx, S_meas, w, alpha, K, Mv=Mv)[0]
            fd = (fp - fm) / (2 * h)
            assert abs(fd - comp) <= 1e-6 * np.abs(grad).max(), (v, direction, fd, comp)


def test_normalised_weights_and_penalty_value():
    S = np.array([[1.0 + 1.0j, 0.5], [0.25j, -2.0]])
    assert np.allclose(p1.normalised_weights(S), [[0.5, 4.0], [16.0, 0.25]])
    mesh = cube_mesh(2)
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    kap = np.full(mesh.nv, 3.0 - 1.0j)
    R, gR = p1.regularisation(K, kap, 0.7)
    assert abs(R) <= 1e-14 and np.abs(gR).max() <= 1e-13
