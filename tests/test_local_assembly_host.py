"""Host logic of the local operators B_i and of the front assembly without a
GPU: the library's maps, through the host-only entry points
mwi_local_assembly_host, mwi_decomposition_host and mwi_fronts_host, against
the oracle's local matrices (Section 3: the form of Eq. pbdirectvarf on
T_i^delta with the impedance condition on its boundary).

* summing the oracle's element and face matrices over every stored entry's
  contributions, in the library's order, gives the oracle's B_i (<= 1e-14 of
  max |B_i|), and each contribution's DOFs are the entry's;
* the front assembly map sends every entry (v, w), w >= v, of B_i exactly once
  to the front whose pivots hold v, at pivot column v and front row w, and
  never an entry below the diagonal;
for order 1 on the chamber and order 2 on the cube.
"""

import numpy as np
import pytest

import oracle as O
from oracle import dd
from oracle.constants import k0_of
from oracle.topology import LOCAL_FACES
from synthetic import chamber_eps, chamber_mesh, cube_eps, cube_mesh
from tests._helpers import FREQ, key_perm, unpack_pairs

mwi = pytest.importorskip("paper_1607_02573_gb300.mwi")

FACE_FLAG = 1 << 62


@pytest.mark.parametrize("case,order,n_sub", [("chamber", 1, 4), ("cube", 2, 3)])
def test_local_assembly_and_front_maps(case, order, n_sub):
    if case == "chamber":
        mesh = chamber_mesh(8, 7)
        eps = chamber_eps(mesh.xyz, mesh.tet)
    else:
        mesh = cube_mesh(3)
        eps = cube_eps(mesh.xyz, mesh.tet)
    eps = np.asarray(eps)
    dl = mwi.decomposition_host(mesh, n_sub, order=order)
    fh = mwi.fronts_host(mesh, n_sub, order=order)
    info, u_off, urows = fh["info"], fh["u_off"], fh["urows"]
    la = mwi.local_assembly_host(mesh, n_sub, order=order)
    td = mwi.slots_host(mesh, order)["tet_dofs"]
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    perm = key_perm(dl["kind"], dl["verts"], topo)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, dl["part"], 1)
    Bs = dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ)

    k0 = k0_of(FREQ)
    K, M = O.element_matrices(mesh.xyz, topo)
    vol = K.astype(np.complex128) - (k0 * k0) * eps[:, None, None] * M
    fu_tet = dl["fu_tet"].astype(np.int64)
    lf = np.array([next(f for f in range(4) if set(topo.tv[t, LOCAL_FACES[f]].tolist()) == set(v.tolist()))
                   for v, t in zip(dl["fu_verts"], fu_tet)], dtype=np.int64)
    face = 1j * (k0 * np.sqrt(eps[fu_tet]))[:, None, None] * O.face_matrix(mesh.xyz, topo, fu_tet, lf)
    fu_local = np.array([[list(td[t]).index(d) if d >= 0 else -1 for d in fd]
                         for t, fd in zip(fu_tet, la["fu_dofs"])]).reshape(fu_tet.size, -1)
    tab_t, tab_f = unpack_pairs(topo.nl), unpack_pairs(la["fu_dofs"].shape[1])

    rp, col = la["B_row_ptr"], la["B_col"]
    slot_row = np.repeat(np.arange(rp.size - 1), np.diff(rp))
    sp, contrib = la["B_slot_ptr"], la["B_contrib"]
    for i in range(n_sub):
        a, b = dl["sub_off"][i], dl["sub_off"][i + 1]
        glob = dl["loc2glob"][a:b]                      # local ND index -> library DOF
        oi = np.searchsorted(dec.R[i], perm[glob])      # local ND index -> row of the oracle's B_i
        Bi = Bs[i].tocsr()
        fu_lo, fu_hi = dl["fu_off"][i], dl["fu_off"][i + 1]
        qs = np.arange(rp[a], rp[b])
        vals = np.zeros(qs.size, dtype=np.complex128)
        for q in qs:
            v, w = slot_row[q] - a, col[q]
            acc = 0j
            for code in contrib[sp[q]:sp[q + 1]].tolist():
                ent = (code & (FACE_FLAG - 1)) >> 16
                pair = code & 0xFFFF
                if code & FACE_FLAG:
                    assert fu_lo <= ent < fu_hi
                    x, y = tab_f[pair]
                    d = {int(la["fu_dofs"][ent, x]), int(la["fu_dofs"][ent, y])}
                    acc += face[ent, fu_local[ent, x], fu_local[ent, y]]
                else:
                    x, y = tab_t[pair]
                    assert dec.Td[i][ent]
                    d = {int(td[ent, x]), int(td[ent, y])}
                    acc += vol[ent, x, y]
                assert d == {int(glob[v]), int(glob[w])}
            vals[q - rp[a]] = acc
        ref = Bi[oi[slot_row[qs] - a], oi[col[qs]]].A1
        assert np.abs(vals - ref).max() <= 1e-14 * abs(Bi).max(), i
        # every stored nonzero of the oracle's B_i is in the library's pattern
        n_i = b - a
        pat = set(zip((slot_row[rp[a]:rp[b]] - a).tolist(), col[rp[a]:rp[b]].tolist()))
        inv = np.empty(n_i, dtype=np.int64)
        inv[oi] = np.arange(n_i)
        Bc = Bi.tocoo()
        assert set(zip(inv[Bc.row].tolist(), inv[Bc.col].tolist())) <= pat

    # the front assembly map
    fsz = info[:, 2] + info[:, 3]
    f_off = np.concatenate([[0], np.cumsum(fsz.astype(np.int64) * info[:, 2])])[:-1]
    used = np.zeros(col.size, dtype=np.int64)
    afp, aslot, apos = la["amap_front_ptr"], la["amap_slot"], la["amap_pos"]
    for k in range(info.shape[0]):
        sub, start, p, u, _ = info[k]
        a = dl["sub_off"][sub]
        rows = np.concatenate([np.arange(start, start + p), urows[u_off[k]:u_off[k] + u]])
        for q, pos in zip(aslot[afp[k]:afp[k + 1]], apos[afp[k]:afp[k + 1]]):
            rel = pos - f_off[k]
            ci, ri = rel // fsz[k], rel % fsz[k]
            v, w = slot_row[q] - a, col[q]
            assert 0 <= rel < fsz[k] * p and ci < p
            assert rows[ci] == v and rows[ri] == w and w >= v
            used[q] += 1
    upper = col >= (slot_row - dl["sub_off"][np.searchsorted(dl["sub_off"], slot_row, side="right") - 1])
    assert np.all(used[upper] == 1) and np.all(used[~upper] == 0)
