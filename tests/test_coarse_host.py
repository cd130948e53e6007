"""Host logic of the two-level ORAS without a GPU: the library's prolongation
(the midpoint rule of the coarse Whitney fields on the fine edges, with its
point location) against the oracle's CoarseSpace, through the host-only entry
point mwi_coarse_prolongation_host.

* a jittered, permuted fine chamber on an unjittered coarse one, whose
  staircase boundary leaves fine midpoints outside the coarse mesh: P agrees
  entry by entry (<= 1e-12 of max |P|);
* two meshes of the impedance cube: the same;
* the fine mesh as its own coarse mesh: P is the identity;
* a second-order fine mesh: only its Whitney DOFs get rows, and those rows are
  the first-order prolongation's.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import dd
from synthetic import chamber_mesh, cube_mesh
from tests._helpers import key_perm

mwi = pytest.importorskip("paper_1607_02573_gb300.mwi")


def _perm_matrix(perm):
    n = perm.size
    return sp.csr_matrix((np.ones(n), (np.arange(n), perm)), shape=(n, n))


def _oracle_p(fine, coarse):
    ft = O.build_topology(fine.tet, fine.bface_tag, fine.nv, 1)
    ct = O.build_topology(coarse.tet, coarse.bface_tag, coarse.nv, 1)
    # the oracle's CoarseSpace also factorises P^T A P; with A = I that is P^T P
    A = sp.identity(ft.ndof, format="csr", dtype=np.complex128)
    return dd.CoarseSpace(fine.xyz, ft, coarse.xyz, ct, A, None).P, ft, ct


def _lib_in_oracle_order(fine, coarse, ft, ct):
    P, (fk, fv), (ck, cv) = mwi.coarse_prolongation_host(fine, coarse)
    Pf, Pc = _perm_matrix(key_perm(fk, fv, ft)), _perm_matrix(key_perm(ck, cv, ct))
    return (Pf.T @ P @ Pc).tocsr()


@pytest.mark.parametrize("fine,coarse", [((10, 9), (6, 5)), ((12, 11), (5, 4))])
def test_chamber_prolongation_matches_oracle(fine, coarse):
    fm = chamber_mesh(*fine)
    cm = chamber_mesh(*coarse, jitter=0.0, permute=False)
    Po, ft, ct = _oracle_p(fm, cm)
    Pl = _lib_in_oracle_order(fm, cm, ft, ct)
    assert abs(Pl - Po).max() <= 1e-12 * abs(Po).max()
    assert Pl.nnz >= 0.99 * Po.nnz


def test_cube_prolongation_matches_oracle():
    fm, cm = cube_mesh(5), cube_mesh(3)
    Po, ft, ct = _oracle_p(fm, cm)
    Pl = _lib_in_oracle_order(fm, cm, ft, ct)
    assert abs(Pl - Po).max() <= 1e-12 * abs(Po).max()


def test_self_prolongation_is_identity():
    m = chamber_mesh(8, 7)
    P, (fk, fv), (ck, cv) = mwi.coarse_prolongation_host(m, m)
    assert np.array_equal(fk, ck) and np.array_equal(fv, cv)
    assert abs(P - sp.identity(P.shape[0])).max() <= 1e-12


def test_second_order_fine_mesh_rows():
    fm = chamber_mesh(8, 7)
    cm = chamber_mesh(5, 4, jitter=0.0, permute=False)
    P2, (fk, fv), (ck, cv) = mwi.coarse_prolongation_host(fm, cm, 2)
    P1, (gk, gv), _ = mwi.coarse_prolongation_host(fm, cm, 1)
    whit = fk == 0
    assert np.all(np.diff(P2.indptr)[~whit] == 0)
    # the Whitney rows of the second-order mesh are the first-order rows, matched by DOF key
    key2 = {(int(a), int(b)): i for i, (a, b) in enumerate(fv[whit][:, :2])}
    rows2 = np.nonzero(whit)[0]
    order = np.array([rows2[key2[(int(a), int(b))]] for a, b in gv[:, :2]])
    assert abs(P2[order] - P1).max() == 0.0
