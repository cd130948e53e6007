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


def _elimination_structure(n, adj):
    """struct(L[:, k]) of the LDL^T factor of a matrix with the symmetric
    graph adj (lists of neighbours, no self loops) eliminated in the order
    0..n-1: the neighbours above k plus the structures of k's children in the
    elimination tree (Liu's row-merge form of symbolic factorisation)."""
    kids = [[] for _ in range(n)]
    out = []
    for k in range(n):
        s = {j for j in adj[k] if j > k}
        for c in kids[k]:
            s |= out[c]
        s.discard(k)
        out.append(s)
        if s:
            kids[min(s)].append(k)
    return out


@pytest.mark.parametrize("case,order,n_sub,leaf", [("chamber", 1, 4, 16), ("cube", 2, 2, 32)])
def test_fronts_cover_the_elimination_fill(case, order, n_sub, leaf):
    """The multifrontal structure of every subdomain: the fronts' pivots tile
    the local rows; a front's update rows are ancestors' pivots, ascending, and
    lie in its parent's front (the extend-add's premise); the root fronts have
    none; and every column's fill in the exact symbolic LDL^T of the graph of
    B_i (DOFs coupled through a tet of T_i^delta) in the nested-dissection
    order lies in the rows of the column's front."""
    mesh = chamber_mesh(10, 9) if case == "chamber" else cube_mesh(4)
    lib = mwi.decomposition_host(mesh, n_sub, nd_leaf=leaf, order=order)
    fh = mwi.fronts_host(mesh, n_sub, nd_leaf=leaf, order=order)
    info, u_off, urows = fh["info"], fh["u_off"], fh["urows"]
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    perm = key_perm(lib["kind"], lib["verts"], topo)
    part = dd.rcb_partition(mesh.xyz, mesh.tet, n_sub)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    for i in range(n_sub):
        a, b = lib["sub_off"][i], lib["sub_off"][i + 1]
        n = b - a
        g2l = -np.ones(topo.ndof, dtype=np.int64)
        g2l[perm[lib["loc2glob"][a:b]]] = np.arange(n)
        adj = [set() for _ in range(n)]
        for t in np.nonzero(dec.Td[i])[0]:
            d = topo.tet_dofs[t]
            loc = g2l[d[d >= 0]]
            for x in loc:
                adj[x].update(loc.tolist())
        for k in range(n):
            adj[k].discard(k)
        fill = _elimination_structure(n, adj)
        ids = np.nonzero(info[:, 0] == i)[0]
        fr = info[ids]
        order_ = np.argsort(fr[:, 1])
        starts, ps = fr[order_, 1], fr[order_, 2]
        assert starts[0] == 0 and np.array_equal(starts[1:], (starts + ps)[:-1]) and starts[-1] + ps[-1] == n
        rows_of = {}
        for f, (sub, start, p, u, parent) in zip(ids, fr):
            U = urows[u_off[f]:u_off[f] + u]
            assert np.all(np.diff(U) > 0) and (u == 0 or U[0] >= start + p)
            rows_of[f] = (start, p, set(U.tolist()))
            if parent < 0:
                assert u == 0
            else:
                assert parent > f and info[parent, 0] == i
        for f, (start, p, U) in rows_of.items():
            parent = info[f, 4]
            if parent >= 0:
                ps_, pp, pU = rows_of[parent]
                assert U <= set(range(ps_, ps_ + pp)) | pU
                # urel: each update row's position among the parent's front rows
                prow = list(range(ps_, ps_ + pp)) + sorted(pU)
                Ul = urows[u_off[f]:u_off[f] + info[f, 3]].tolist()
                assert fh["urel"][u_off[f]:u_off[f] + info[f, 3]].tolist() == [prow.index(x) for x in Ul]
            front_rows = set(range(start, start + p)) | U
            for k in range(start, start + p):
                assert fill[k] <= front_rows, (i, f, k)
    # the sweeps' extend-add table: front row t of front s gathers, children
    # ascending, the update-buffer rows of its children's update rows at t
    f = info[:, 2].astype(np.int64) + info[:, 3]
    base = np.concatenate([[0], np.cumsum(f)])
    upd = np.concatenate([[0], np.cumsum(info[:, 3].astype(np.int64))])
    want = [[] for _ in range(int(base[-1]))]
    for c in range(info.shape[0]):
        s_ = info[c, 4]
        if s_ < 0:
            continue
        for j in range(info[c, 3]):
            want[base[s_] + fh["urel"][u_off[c] + j]].append(int(upd[c] + j))
    ap, src = fh["asm_ptr"], fh["asm_src"]
    assert ap.size == base[-1] + 1
    for r in range(int(base[-1])):
        assert src[ap[r]:ap[r + 1]].tolist() == want[r]
