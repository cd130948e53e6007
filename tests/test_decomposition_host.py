"""Host logic of the ORAS decomposition (Section 3) without a GPU: the
library's partition, overlap, partition of unity and boundary face uses,
through the host-only entry point mwi_decomposition_host, against the
oracle's Decomposition and against the definitions.

* the partition is the oracle's recursive coordinate bisection, tet for tet;
* each subdomain's local rows are the DOFs of T_i^delta (the oracle's R_i),
  each once, and its weights are the oracle's D_i (Eq. chi at the DOF);
* sum_i R_i^T D_i R_i = I (Eq. algebPartUnity) at every DOF when the overlap
  is at least one layer;
* the face uses of B_i are, by definition, the non-PEC faces with exactly one
  tet in T_i^delta, owned by that tet;
for overlaps 0, 1 and 2, order 1 and 2, chamber and cube.
"""

import numpy as np
import pytest

import oracle as O
from oracle import dd
from synthetic import chamber_mesh, cube_mesh
from tests._helpers import key_perm

mwi = pytest.importorskip("paper_1607_02573_gb300.mwi")


@pytest.mark.parametrize("case,order,n_sub,overlap", [("chamber", 1, 4, 1), ("chamber", 1, 8, 2),
                                                      ("chamber", 2, 4, 1), ("cube", 1, 6, 0),
                                                      ("cube", 2, 3, 2)])
def test_decomposition_matches_oracle(case, order, n_sub, overlap):
    mesh = chamber_mesh(10, 9) if case == "chamber" else cube_mesh(5)
    lib = mwi.decomposition_host(mesh, n_sub, overlap=overlap if overlap > 0 else -1, order=order)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    perm = key_perm(lib["kind"], lib["verts"], topo)
    part = dd.rcb_partition(mesh.xyz, mesh.tet, n_sub)
    assert np.array_equal(lib["part"], part)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, overlap)
    total = np.zeros(topo.ndof)
    for i in range(n_sub):
        a, b = lib["sub_off"][i], lib["sub_off"][i + 1]
        rows = perm[lib["loc2glob"][a:b]]
        assert np.array_equal(np.sort(rows), dec.R[i])  # the DOFs of T_i^delta, each once
        want = dec.D[i][np.searchsorted(dec.R[i], rows)]
        assert np.abs(lib["dweight"][a:b] - want).max() <= 1e-15
        np.add.at(total, rows, lib["dweight"][a:b])
        # boundary face uses of T_i^delta, from the definition
        td = dec.Td[i]
        ft = topo.face_tets
        ina = (ft[:, 0] >= 0) & td[np.maximum(ft[:, 0], 0)]
        inb = (ft[:, 1] >= 0) & td[np.maximum(ft[:, 1], 0)]
        sel = np.nonzero((ina ^ inb) & (topo.face_tag != 1))[0]
        owner = np.where(ina[sel], ft[sel, 0], ft[sel, 1])
        want_fu = {(tuple(topo.faces[f]), int(t)) for f, t in zip(sel, owner)}
        a, b = lib["fu_off"][i], lib["fu_off"][i + 1]
        got_fu = {(tuple(v), int(t)) for v, t in zip(lib["fu_verts"][a:b].tolist(), lib["fu_tet"][a:b])}
        assert b - a == len(got_fu) and got_fu == want_fu
    if overlap >= 1:  # with no overlap the weights of a subdomain that touches only an edge's end do not vanish
        assert np.abs(total - 1.0).max() <= 1e-14
    nloc = lib["sub_off"][-1]
    assert nloc <= lib["factor_entries"] <= sum(int(len(r)) ** 2 for r in dec.R)


def test_bad_decomposition_arguments_are_refused():
    mesh = cube_mesh(2)
    with pytest.raises(mwi.MwiError, match="MWI_EINVAL"):
        mwi.decomposition_host(mesh, 10 ** 6)
    with pytest.raises(mwi.MwiError, match="MWI_EINVAL"):
        mwi.decomposition_host(mesh, 4, overlap=9)
