"""Host logic of the atomic-free assembly of A (Eq. pbdirectvarf, Eq. linsys)
without a GPU: the library's slot map, through the host-only entry point
mwi_slots_host, against the oracle's assembly.

* every tet's local DOFs are the oracle's, in the oracle's local order;
* the CSR pattern is the DOF pairs sharing a tet: the oracle's nonzeros and
  entries that cancel to exactly zero;
* every contribution of a stored entry (r, c) is an element pair (tet, i, j)
  or a face-use pair whose DOFs are {r, c}; every element pair with two live
  DOFs, and every impedance face-use pair, appears in exactly the entries it
  couples; the mirrored entry (c, r) lists the same contributions in the
  same order (so the device sums give a bit-for-bit symmetric A);
* the face uses are the impedance faces with their owning tets;
* summing the oracle's element matrices over the contributions, in the
  library's order, reproduces the oracle's A (<= 1e-14 of max |A|);
for order 1 and 2, chamber (PEC and impedance faces) and cube.
"""

import numpy as np
import pytest

import oracle as O
from oracle.assemble import impedance_faces
from oracle.constants import k0_of
from oracle.topology import LOCAL_FACES
from synthetic import chamber_eps, chamber_mesh, cube_eps, cube_mesh
from tests._helpers import FREQ, key_perm, unpack_pairs

mwi = pytest.importorskip("paper_1607_02573_gb300.mwi")

FACE_FLAG = 1 << 62


@pytest.mark.parametrize("case,order", [("chamber", 1), ("chamber", 2), ("cube", 1), ("cube", 2)])
def test_slot_map_reproduces_the_oracle_assembly(case, order):
    if case == "chamber":
        mesh = chamber_mesh(7, 6)
        eps = chamber_eps(mesh.xyz, mesh.tet)
    else:
        mesh = cube_mesh(3)
        eps = cube_eps(mesh.xyz, mesh.tet)
    lib = mwi.slots_host(mesh, order)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    perm = key_perm(lib["kind"], lib["verts"], topo)
    nl = topo.nl
    td = lib["tet_dofs"]
    assert np.array_equal(np.where(td >= 0, perm[np.maximum(td, 0)], -1), topo.tet_dofs)

    A = O.assemble_system(mesh.xyz, topo, eps, FREQ).tocsr()
    rp, col = lib["row_ptr"], lib["col"]
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    got = set(zip(perm[rows].tolist(), perm[col].tolist()))
    Acoo = A.tocoo()
    # the library's pattern is structural (DOF pairs sharing a tet); the oracle's
    # sparse sum drops entries that cancel to exactly zero, which the value
    # check below finds zero in the library's sums too
    assert set(zip(Acoo.row.tolist(), Acoo.col.tolist())) <= got and len(got) == col.size

    # face uses: the impedance faces and their owners
    ft, fl = impedance_faces(topo)
    want_fu = {(tuple(topo.faces[topo.tet_faces[t, f]]), int(t)) for t, f in zip(ft, fl)}
    got_fu = {(tuple(v), int(t)) for v, t in zip(lib["fu_verts"].tolist(), lib["fu_tet"])}
    assert len(got_fu) == lib["fu_tet"].size and got_fu == want_fu

    # element matrices in the oracle's local order; face matrices over the owner's local DOFs
    K, M = O.element_matrices(mesh.xyz, topo)
    k0 = k0_of(FREQ)
    vol = K.astype(np.complex128) - (k0 * k0) * np.asarray(eps)[:, None, None] * M
    lf = np.empty(lib["fu_tet"].size, dtype=np.int64)
    for u, (v, t) in enumerate(zip(lib["fu_verts"], lib["fu_tet"])):
        lf[u] = next(f for f in range(4) if set(topo.tv[t, LOCAL_FACES[f]].tolist()) == set(v.tolist()))
    Bf = O.face_matrix(mesh.xyz, topo, lib["fu_tet"].astype(np.int64), lf)
    face = 1j * (k0 * np.sqrt(np.asarray(eps)[lib["fu_tet"]]))[:, None, None] * Bf
    fu_local = np.array([[list(td[t]).index(d) if d >= 0 else -1 for d in fd]
                         for t, fd in zip(lib["fu_tet"], lib["fu_dofs"])]).reshape(lib["fu_tet"].size, -1)

    tab_t, tab_f = unpack_pairs(nl), unpack_pairs(lib["fu_dofs"].shape[1])
    sp, contrib = lib["slot_ptr"], lib["contrib"]
    seen = {}
    lists = {}
    val = np.zeros(col.size, dtype=np.complex128)
    for q in range(col.size):
        r, c = int(rows[q]), int(col[q])
        lst = contrib[sp[q]:sp[q + 1]].tolist()
        lists[(r, c)] = lst
        acc = 0j
        for code in lst:
            is_face = bool(code & FACE_FLAG)
            ent = (code & (FACE_FLAG - 1)) >> 16
            pair = code & 0xFFFF
            if is_face:
                i, j = tab_f[pair]
                d = (int(lib["fu_dofs"][ent, i]), int(lib["fu_dofs"][ent, j]))
                li, lj = fu_local[ent, i], fu_local[ent, j]
                acc += face[ent, li, lj]
            else:
                i, j = tab_t[pair]
                d = (int(td[ent, i]), int(td[ent, j]))
                acc += vol[ent, i, j]
            assert sorted(d) == sorted((r, c)), (q, code)
            key = (is_face, ent, i, j)
            seen[key] = seen.get(key, 0) + 1
        val[q] = acc
    # every element / face-use pair with two live DOFs, in each entry it couples once
    for t in range(topo.nt):
        for i in range(nl):
            for j in range(i, nl):
                if td[t, i] >= 0 and td[t, j] >= 0:
                    assert seen.get((False, t, i, j), 0) == (1 if i == j else 2)
    fd = lib["fu_dofs"]
    for u in range(fd.shape[0]):
        for i in range(fd.shape[1]):
            for j in range(i, fd.shape[1]):
                if fd[u, i] >= 0 and fd[u, j] >= 0:
                    assert seen.get((True, u, i, j), 0) == (1 if i == j else 2)
    assert sum(seen.values()) == contrib.size
    # mirrored entries: the same contributions in the same order
    for (r, c), lst in lists.items():
        assert lists[(c, r)] == lst
    # the sums reproduce the oracle's A
    Ad = A[perm[rows], perm[col]].A1
    assert np.abs(val - Ad).max() <= 1e-14 * np.abs(Ad).max()
