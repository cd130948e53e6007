"""Pins for the oracle's P1 parameter, gradient penalty and normalised weights
(Eq. defJ2, the P1 parameter of Section 6.3).

* the P1 stiffness matrix annihilates constants, is symmetric positive
  semidefinite, and gives |a|^2 times the volume for a linear field a.x + b;
* spreading per-tet values to the vertices is the adjoint of the centroid
  sampling for the real inner product;
* the gradient of the full objective (normalised misfit + penalty) equals
  central finite differences in Re and Im of kappa at sampled vertices.
"""

import numpy as np

import oracle as O
from oracle import p1
from synthetic import antenna_array, chamber_mesh, cube_antennas, cube_mesh

FREQ = 1e9


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


def test_spread_is_adjoint_of_centroid_sampling():
    mesh = cube_mesh(4)
    rng = np.random.default_rng(2)
    kap = rng.standard_normal(mesh.nv) + 1j * rng.standard_normal(mesh.nv)
    g = rng.standard_normal(mesh.nt) + 1j * rng.standard_normal(mesh.nt)
    lhs = np.real(np.vdot(p1.p1_to_tet(mesh.tet, kap), g))
    rhs = np.real(np.vdot(kap, p1.p1_spread(mesh.tet, mesh.nv, g)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_objective_gradient_matches_finite_differences():
    mesh = cube_mesh(4)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    tx = antenna_array(cube_antennas())
    rng = np.random.default_rng(3)
    kap_true = 44 - 20j + rng.uniform(-6, 6, mesh.nv) + 1j * rng.uniform(-3, 3, mesh.nv)
    w = p1.empty_chamber_weights(mesh.xyz, topo, np.full(mesh.nt, 44 - 20j), FREQ, tx, tx)
    S_meas = O.forward(mesh.xyz, topo, p1.p1_to_tet(mesh.tet, kap_true), FREQ, tx, tx)["S"]
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    alpha = 1e-3
    kap = np.full(mesh.nv, 44 - 20j) + rng.uniform(-1, 1, mesh.nv)
    phi, grad = p1.objective_p1(mesh.xyz, topo, mesh.tet, kap, FREQ, tx, tx, S_meas, w, alpha, K)
    assert phi > 0
    for v in rng.choice(mesh.nv, 4, replace=False):
        for direction, comp in ((1.0, grad[v].real), (1j, grad[v].imag)):
            h = 1e-5 * abs(kap[v])
            kp = kap.copy(); kp[v] += direction * h
            km = kap.copy(); km[v] -= direction * h
            fp = p1.objective_p1(mesh.xyz, topo, mesh.tet, kp, FREQ, tx, tx, S_meas, w, alpha, K)[0]
            fm = p1.objective_p1(mesh.xyz, topo, mesh.tet, km, FREQ, tx, tx, S_meas, w, alpha, K)[0]
            fd = (fp - fm) / (2 * h)
            assert abs(fd - comp) <= 1e-5 * np.abs(grad).max(), (v, direction, fd, comp)


def test_normalised_weights_and_penalty_value():
    S = np.array([[1.0 + 1.0j, 0.5], [0.25j, -2.0]])
    assert np.allclose(p1.normalised_weights(S), [[0.5, 4.0], [16.0, 0.25]])
    mesh = cube_mesh(2)
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    kap = np.full(mesh.nv, 3.0 - 1.0j)
    R, gR = p1.regularisation(K, kap, 0.7)
    assert abs(R) <= 1e-14 and np.abs(gR).max() <= 1e-13
