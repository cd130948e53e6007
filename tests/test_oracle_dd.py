"""Pins for the oracle's ORAS preconditioner and FGMRES (Section 3, Eq. ORAS).

* partition of unity: sum_i R_i^T D_i R_i = I (Eq. algebPartUnity) and
  sum_i chi_i = 1 at every node (Eq. chi);
* with one subdomain, B_1 = A and M^{-1} = A^{-1}: FGMRES stops after one step;
* each B_i is complex symmetric and agrees with A on the rows of DOFs whose
  every tet lies inside T_i^delta (the interface term only touches the rim);
* each B_i is the global assembly (Eq. pbdirectvarf with its outer impedance
  condition, whose sign the outgoing-datum test pins) run on the submesh
  T_i^delta alone, with the faces it shares with the rest of the domain
  tagged as impedance faces: the interface term has the outer condition's
  sign, the owner tet's wavenumber and exactly those faces (order 1 and 2,
  delta 1 and 2, chamber and cube);
* FGMRES + ORAS reaches the direct solution;
* the RCB partition covers every tet once and is balanced.
"""

import numpy as np
import pytest

import oracle as O
from oracle import dd
from synthetic import antenna_array, chamber_eps, chamber_mesh, cube_eps, cube_mesh, ring_antennas

FREQ = 1e9


@pytest.fixture(scope="module")
def small_chamber():
    mesh = chamber_mesh(10, 9)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ)
    return mesh, topo, eps, A


def test_rcb_partition_balanced(small_chamber):
    mesh, *_ = small_chamber
    for p in (1, 2, 5, 8):
        part = dd.rcb_partition(mesh.xyz, mesh.tet, p)
        cnt = np.bincount(part, minlength=p)
        assert cnt.sum() == mesh.nt and cnt.min() >= mesh.nt // p - 1 and cnt.max() <= mesh.nt // p + 2


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("nsub,delta", [(4, 1), (8, 2)])
def test_partition_of_unity_identity(small_chamber, order, nsub, delta):
    mesh = small_chamber[0]
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    part = dd.rcb_partition(mesh.xyz, mesh.tet, nsub)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, delta)
    assert np.abs(dec.chi.sum(axis=0) - 1.0).max() <= 1e-15
    acc = np.zeros(topo.ndof)
    for R, D in zip(dec.R, dec.D):
        np.add.at(acc, R, D)
    assert np.abs(acc - 1.0).max() <= 2.3e-16 * 4


def test_single_subdomain_is_exact(small_chamber):
    mesh, topo, eps, A = small_chamber
    part = np.zeros(mesh.nt, dtype=np.int64)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    (B,) = dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ)
    assert abs(B - A).max() <= 1e-12 * abs(A).max()
    oras = dd.ORAS(dec, [B])
    b = np.zeros(topo.ndof, dtype=np.complex128)
    b[5] = 1.0
    x, it, _ = dd.fgmres(A, b, oras.apply, rtol=1e-10)
    assert it == 1


def test_local_matrices_symmetric_and_interior_rows(small_chamber):
    mesh, topo, eps, A = small_chamber
    part = dd.rcb_partition(mesh.xyz, mesh.tet, 4)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    Bs = dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ)
    A = A.tocsr()
    for i, B in enumerate(Bs):
        assert abs(B - B.T).max() == 0.0
        # DOFs all of whose tets lie in T_i^delta: B_i row equals A row restricted
        R = dec.R[i]
        outside = ~dec.Td[i]
        touched = np.zeros(topo.ndof + 1, dtype=bool)
        d = topo.tet_dofs[outside].ravel()
        touched[d[d >= 0]] = True
        inner = np.nonzero(~touched[R])[0]
        Ar = A[R[inner]][:, R]
        assert abs(Ar - B.tocsr()[inner]).max() <= 1e-12 * abs(A).max()
        # rim rows differ (interface impedance and missing outside tets)
        assert inner.size < R.size


def _dof_keys(topo):
    v = topo.dof_verts.astype(np.int64) + 1
    n = topo.nv + 1
    return ((topo.dof_kind.astype(np.int64) * n + v[:, 0]) * n + v[:, 1]) * n + v[:, 2]


def _submesh_system(mesh, eps, tets, order):
    """assemble_system on the tets `tets` alone; faces they share with other
    tets of the mesh become impedance faces, the others keep their tags."""
    tet = np.asarray(mesh.tet, dtype=np.int64)
    opp = [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]  # face opposite local vertex k

    def face_keys(t):
        f = np.sort(t[:, opp], axis=2)
        return (f[:, :, 0] * mesh.nv + f[:, :, 1]) * mesh.nv + f[:, :, 2]

    all_keys, cnt_all = np.unique(face_keys(tet), return_counts=True)
    sk = face_keys(tet[tets])
    sub_keys, cnt_sub = np.unique(sk, return_counts=True)
    shared = cnt_all[np.searchsorted(all_keys, sub_keys)] == 2
    interface = sub_keys[shared & (cnt_sub == 1)]
    tag = np.asarray(mesh.bface_tag, dtype=np.int64)[tets].copy()
    tag[np.isin(sk, interface)] = 2
    topo_s = O.build_topology(tet[tets], tag, mesh.nv, order)
    return topo_s, O.assemble_system(mesh.xyz, topo_s, eps[tets], FREQ).tocsr()


@pytest.mark.parametrize("case,order,delta", [("chamber", 1, 1), ("chamber", 2, 1), ("chamber", 1, 2),
                                              ("cube", 1, 1), ("cube", 2, 2)])
def test_local_matrix_is_submesh_problem_with_impedance_interface(case, order, delta):
    if case == "chamber":
        mesh = chamber_mesh(8, 7)
        eps = chamber_eps(mesh.xyz, mesh.tet)
    else:
        mesh = cube_mesh(4)
        eps = cube_eps(mesh.xyz, mesh.tet)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    part = dd.rcb_partition(mesh.xyz, mesh.tet, 4)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, delta)
    Bs = dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ)
    kg = _dof_keys(topo)
    for i, B in enumerate(Bs):
        topo_s, As = _submesh_system(mesh, eps, np.nonzero(dec.Td[i])[0], order)
        ks = _dof_keys(topo_s)
        # DOFs of R_i in the submesh numbering; the submesh may keep a few more
        # DOFs (edges on PEC faces of tets outside T_i^delta), which the global
        # problem removes: dropping their rows and columns is that removal
        srt = np.argsort(ks)
        pos = np.searchsorted(ks[srt], kg[dec.R[i]])
        assert np.array_equal(ks[srt][pos], kg[dec.R[i]])
        loc = srt[pos]
        Ar = As[loc][:, loc]
        assert abs(Ar - B.tocsr()).max() <= 1e-13 * abs(Ar).max(), i


def test_fgmres_oras_reaches_direct_solution(small_chamber):
    mesh, topo, eps, A = small_chamber
    part = dd.rcb_partition(mesh.xyz, mesh.tet, 8)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    oras = dd.ORAS(dec, dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ))
    ants = antenna_array(ring_antennas(4, radius=0.08))
    tdof, tsgn = O.antenna_edges(mesh.xyz, topo, ants)
    b = O.build_rhs(topo.ndof, tdof, tsgn, np.ones(4), FREQ)
    U_d, _ = O.direct_solve(A, b)
    U, its = dd.solve_oras(A, b, oras, rtol=1e-10)
    for j in range(4):
        assert np.linalg.norm(U[:, j] - U_d[:, j]) <= 1e-8 * np.linalg.norm(U_d[:, j])
        assert np.linalg.norm(A @ U[:, j] - b[:, j]) <= 1e-10 * np.linalg.norm(b[:, j])
    assert max(its) < 60
