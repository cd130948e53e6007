"""Pins for the oracle's solves, S-parameters, misfit and gradient (Sections 4-5).

* the direct solve leaves a residual at rounding level;
* reciprocity: S = S^T because the form is bilinear (A = A^T);
* the adjoint identity, checked as <A^{-1} x, y> = <x, A^{-1} y> (unconjugated);
* the adjoint gradient equals central finite differences of J with respect to
  Re and Im of eps on sampled tets, including tets that own an impedance face,
  for first- and second-order elements;
* J = 0 and grad = 0 when the measurements equal the simulation.
"""

import numpy as np
import pytest

import oracle as O
from synthetic import antenna_array, chamber_mesh, cube_antennas, cube_eps, cube_mesh, ring_antennas

FREQ = 1e9


def _cube_problem(n=4, seed=4, order=1):
    mesh = cube_mesh(n)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    rng = np.random.default_rng(seed)
    eps = 44 - 20j + rng.uniform(-5, 5, mesh.nt) + 1j * rng.uniform(-3, 3, mesh.nt)
    tx = antenna_array(cube_antennas())
    return mesh, topo, eps, tx


def test_direct_residual_and_reciprocity_cube():
    mesh = cube_mesh(8)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    eps = cube_eps(mesh.xyz, mesh.tet)
    tx = antenna_array(cube_antennas())
    f = O.forward(mesh.xyz, topo, eps, FREQ, tx, tx)
    r = f["A"] @ f["U"] - f["b"]
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(f["b"])
    S = f["S"]
    assert np.abs(S - S.T).max() <= 1e-12 * np.abs(S).max()
    # reflection dominates each column (Section 6.2: reflections near 0 dB, transmissions far below)
    assert np.all(np.argmax(np.abs(S), axis=0) == np.arange(4))


def test_reciprocity_chamber_ring():
    mesh = chamber_mesh(11, 10)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    eps = np.full(mesh.nt, 44 - 20j)
    ants = antenna_array(ring_antennas(8, radius=0.1))
    f = O.forward(mesh.xyz, topo, eps, FREQ, ants, ants)
    S = f["S"]
    assert np.abs(S - S.T).max() <= 1e-11 * np.abs(S).max()
    # transmission decays with angular distance from the transmitter in the homogeneous gel
    col = np.abs(S[:, 0])
    assert col[0] > col[1] > col[2] > col[4]


def test_adjoint_dot_identity():
    mesh, topo, eps, _ = _cube_problem()
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(topo.ndof) + 1j * rng.standard_normal(topo.ndof)
    y = rng.standard_normal(topo.ndof) + 1j * rng.standard_normal(topo.ndof)
    U, _ = O.direct_solve(A, np.stack([x, y], 1))
    lhs = U[:, 0] @ y
    rhs = x @ U[:, 1]
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("weighted,order", [(False, 1), (True, 1), (True, 2)])
def test_gradient_matches_finite_differences(weighted, order):
    mesh, topo, eps, tx = _cube_problem(n=4 if order == 1 else 3, order=order)
    f0 = O.forward(mesh.xyz, topo, eps, FREQ, tx, tx)
    rng = np.random.default_rng(1)
    S_meas = f0["S"] * (1 + 0.3 * rng.standard_normal(f0["S"].shape)) + 0.1 * np.abs(f0["S"]).mean()
    w = rng.uniform(0.5, 2.0, S_meas.shape) if weighted else None
    J, grad, _ = O.misfit_and_gradient(mesh.xyz, topo, eps, FREQ, tx, tx, S_meas, w, fwd=f0)
    # sampled tets: largest |grad|, a random interior one and tets owning impedance faces
    owners = np.unique(topo.face_tets[topo.face_tag == 2, 0])
    pick = [int(np.argmax(np.abs(grad))), int(rng.integers(mesh.nt)), int(owners[0]), int(owners[7])]

    K, M = O.element_matrices(mesh.xyz, topo)

    def J_at(e):
        f = O.forward(mesh.xyz, topo, e, FREQ, tx, tx, A=O.assemble_system(mesh.xyz, topo, e, FREQ, K=K, M=M))
        return O.misfit(f["S"], S_meas, w)[0]

    for t in pick:
        for direction, comp in ((1.0, grad[t].real), (1j, grad[t].imag)):
            h = 1e-5 * abs(eps[t])
            ep = eps.copy(); ep[t] += direction * h
            em = eps.copy(); em[t] -= direction * h
            fd = (J_at(ep) - J_at(em)) / (2 * h)
            assert abs(fd - comp) <= 1e-5 * np.abs(grad).max(), (t, direction, fd, comp)


def test_zero_misfit_zero_gradient():
    mesh, topo, eps, tx = _cube_problem()
    f0 = O.forward(mesh.xyz, topo, eps, FREQ, tx, tx)
    J, grad, _ = O.misfit_and_gradient(mesh.xyz, topo, eps, FREQ, tx, tx, f0["S"].copy(), fwd=f0)
    assert J == 0.0
    assert np.abs(grad).max() == 0.0


def test_antenna_edges_on_cube_face_centres():
    mesh = cube_mesh(8)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    tx = antenna_array(cube_antennas())
    d, s = O.antenna_edges(mesh.xyz, topo, tx)
    for k, (dof, sg) in enumerate(zip(d, s)):
        a, b = topo.dof_verts[dof, :2]
        vec = (mesh.xyz[b] - mesh.xyz[a]) * sg
        assert np.allclose(vec / np.linalg.norm(vec), [0, 0, 1])
        start = mesh.xyz[a] if sg > 0 else mesh.xyz[b]
        assert np.allclose(start, tx[k, 0:3])
