"""Pins for the oracle's two-level ORAS (coarse space of Section 7).

* with the fine mesh as its own coarse mesh the prolongation is the identity
  (a Whitney function's tangential integral along its own edge is 1, along the
  other edges 0, and it is constant along an edge, so the midpoint rule is exact);
* the fields a + b x x are reproduced: their coarse DOFs prolong to their
  fine DOFs (lowest-order Whitney elements contain exactly these fields, and
  the midpoint rule is exact for their tangential integrals along an edge),
  on two different meshes of the cube, the fine one jittered, and on a coarse
  chamber whose staircase boundary leaves fine midpoints outside it (the
  affine extension of a tet's interpolant of such a field is the field);
* with the fine mesh as coarse mesh, Q = A^{-1} and the deflated two-level
  preconditioner is exact: FGMRES stops after one step;
* on the chamber, FGMRES with the two-level preconditioner reaches the direct
  solution.
"""

import numpy as np

import oracle as O
from oracle import dd
from synthetic import antenna_array, chamber_eps, chamber_mesh, cube_eps, cube_mesh, ring_antennas

FREQ = 1e9


def _prob(mesh, eps, nsub):
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ).tocsr()
    part = dd.rcb_partition(mesh.xyz, mesh.tet, nsub)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    oras = dd.ORAS(dec, dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ))
    return topo, A, oras


def test_self_prolongation_is_identity_and_two_level_exact():
    mesh = chamber_mesh(8, 7)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    topo, A, oras = _prob(mesh, eps, 4)
    cs = dd.CoarseSpace(mesh.xyz, topo, mesh.xyz, topo, A, oras)
    I = cs.P.toarray()
    assert np.abs(I - np.eye(topo.ndof)).max() <= 1e-12
    b = np.zeros(topo.ndof, dtype=np.complex128)
    b[7] = 1.0
    x, it, _ = dd.fgmres(A, b, cs.apply, rtol=1e-10)
    assert it == 1


def _whitney_dofs(xyz, topo, F):
    """DOFs of the field F(x) (affine in x) on every live Whitney edge:
    F(midpoint) . (x_hi - x_lo), the exact tangential integral."""
    out = np.zeros(topo.ndof)
    e = topo.edges
    d = np.full(e.shape[0], -1, dtype=np.int64)
    d[topo.tet_edges.ravel()] = topo.tet_dofs[:, :6].ravel()
    ok = d >= 0
    mid = 0.5 * (xyz[e[ok, 0]] + xyz[e[ok, 1]])
    out[d[ok]] = np.einsum("nd,nd->n", xyz[e[ok, 1]] - xyz[e[ok, 0]], F(mid))
    return out


def test_rigid_fields_are_reproduced():
    a, b = np.array([0.3, -1.1, 0.7]), np.array([2.0, 0.5, -1.3])
    fields = [lambda x: np.broadcast_to(a, x.shape), lambda x: a + np.cross(b, x)]
    cases = [(cube_mesh(5), cube_mesh(3), cube_eps), (chamber_mesh(9, 8), chamber_mesh(5, 4, jitter=0.0, permute=False),
                                                      chamber_eps)]
    for fine, coarse, epsf in cases:
        ft = O.build_topology(fine.tet, fine.bface_tag, fine.nv, 1)
        ct = O.build_topology(coarse.tet, coarse.bface_tag, coarse.nv, 1)
        A = O.assemble_system(fine.xyz, ft, epsf(fine.xyz, fine.tet), FREQ).tocsr()
        cs = dd.CoarseSpace(fine.xyz, ft, coarse.xyz, ct, A, None)
        for F in fields:
            f = _whitney_dofs(fine.xyz, ft, F)
            g = cs.P @ _whitney_dofs(coarse.xyz, ct, F)
            # PEC edges carry no DOF on either mesh; a fine edge whose coarse tet has a PEC
            # edge loses that coarse DOF, so compare on rows whose coarse DOFs are all live
            rows, tets = cs.located
            full = rows[np.all(ct.tet_dofs[tets, :6] >= 0, axis=1)]
            assert full.size > 0.3 * ft.ndof
            assert np.abs(g - f)[full].max() <= 1e-12 * np.abs(f).max()


def test_two_level_reaches_direct_solution():
    mesh = chamber_mesh(10, 9)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    topo, A, oras = _prob(mesh, eps, 8)
    cm = chamber_mesh(6, 5, jitter=0.0, permute=False)
    ct = O.build_topology(cm.tet, cm.bface_tag, cm.nv, 1)
    cs = dd.CoarseSpace(mesh.xyz, topo, cm.xyz, ct, A, oras)
    tx = antenna_array(ring_antennas(2, radius=0.08))
    d, s = O.antenna_edges(mesh.xyz, topo, tx)
    B = O.build_rhs(topo.ndof, d, s, tx[:, 6] + 1j * tx[:, 7], FREQ)
    U = O.direct_solve(A, B)[0]
    for c in range(B.shape[1]):
        x, it, _ = dd.fgmres(A, B[:, c], cs.apply, rtol=1e-10)
        assert np.linalg.norm(x - U[:, c]) <= 1e-8 * np.linalg.norm(U[:, c])
