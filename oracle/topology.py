"""Mesh entities and degrees of freedom (Section 2.1).

Lowest order (degree 1): one DOF per oriented edge, the circulation of the
field along it.  Edges are oriented from the lower to the higher global vertex
id, and every tetrahedron's vertices are first sorted by global id, so a local
edge (i < j) always has the global orientation and no sign flips are needed.

Second order (hierarchical first-kind, 20 functions per tet): per edge the
Whitney function and the gradient of lambda_a lambda_b; per face (a < b < c)
the two functions lambda_c N_ab and lambda_a N_bc.

DOFs on perfectly conducting faces (E x n = 0, Eq. eqmetal) are removed: the
edges of PEC faces, and for order 2 also the face DOFs of PEC faces.
"""

from dataclasses import dataclass

import numpy as np

# local edges and faces of a tet whose vertices are sorted by global id
LOCAL_EDGES = np.array([[0, 1], [0, 2], [0, 3], [1, 2], [1, 3], [2, 3]])
LOCAL_FACES = np.array([[0, 1, 2], [0, 1, 3], [0, 2, 3], [1, 2, 3]])
OPPOSITE = np.array([3, 2, 1, 0])  # vertex opposite local face f

KIND_WHITNEY, KIND_GRAD, KIND_FACE_A, KIND_FACE_B = 0, 1, 2, 3


@dataclass
class Topology:
    order: int
    nv: int
    tv: np.ndarray          # [nt, 4] tet vertices sorted by global id
    edges: np.ndarray       # [ne, 2] (low, high), lexicographically sorted
    tet_edges: np.ndarray   # [nt, 6] edge ids of LOCAL_EDGES
    faces: np.ndarray       # [nf, 3] sorted vertex triples, lexicographically sorted
    tet_faces: np.ndarray   # [nt, 4] face ids of LOCAL_FACES
    face_tag: np.ndarray    # [nf] 0 interior, 1 PEC, 2 impedance
    face_tets: np.ndarray   # [nf, 2] tets sharing the face (-1 if boundary)
    face_local: np.ndarray  # [nf, 2] local face index in each of those tets
    pec_edge: np.ndarray    # [ne] bool
    tet_dofs: np.ndarray    # [nt, nl] global DOF (-1 for removed PEC DOFs)
    ndof: int
    dof_kind: np.ndarray    # [ndof]
    dof_verts: np.ndarray   # [ndof, 3] global vertex ids (third = -1 for edge DOFs)

    @property
    def nt(self):
        return self.tv.shape[0]

    @property
    def nl(self):
        return 6 if self.order == 1 else 20


def _unique_rows(keys):
    uniq, inv = np.unique(keys, return_inverse=True)
    return uniq, inv.reshape(keys.shape)


def build_topology(tet, bface_tag, nv, order=1):
    tet = np.asarray(tet, dtype=np.int64)
    tag_in = np.asarray(bface_tag, dtype=np.int64)
    nt = tet.shape[0]
    srt = np.argsort(tet, axis=1, kind="stable")
    tv = np.take_along_axis(tet, srt, axis=1)
    # tag of the face opposite original local vertex k moves with that vertex
    tag_sorted_vertex = np.take_along_axis(tag_in, srt, axis=1)  # tag of face opposite sorted vertex
    # face f of LOCAL_FACES is opposite sorted vertex OPPOSITE[f]
    tet_face_tag = tag_sorted_vertex[:, OPPOSITE]

    ev = tv[:, LOCAL_EDGES]  # [nt, 6, 2]
    ekeys = ev[:, :, 0] * nv + ev[:, :, 1]
    euniq, tet_edges = _unique_rows(ekeys)
    edges = np.stack([euniq // nv, euniq % nv], axis=1)

    fv = tv[:, LOCAL_FACES]  # [nt, 4, 3]
    fkeys = (fv[:, :, 0] * nv + fv[:, :, 1]) * nv + fv[:, :, 2]
    funiq, tet_faces = _unique_rows(fkeys)
    nf = funiq.size
    faces = np.stack([funiq // (nv * nv), (funiq // nv) % nv, funiq % nv], axis=1)

    face_tag = np.zeros(nf, dtype=np.int64)
    flat_f = tet_faces.ravel()
    flat_tag = tet_face_tag.ravel()
    np.maximum.at(face_tag, flat_f, flat_tag)
    face_tets = -np.ones((nf, 2), dtype=np.int64)
    face_local = -np.ones((nf, 2), dtype=np.int64)
    tidx = np.repeat(np.arange(nt), 4)
    lidx = np.tile(np.arange(4), nt)
    order_f = np.argsort(flat_f, kind="stable")
    sf = flat_f[order_f]
    first = np.ones(sf.size, dtype=bool)
    first[1:] = sf[1:] != sf[:-1]
    slot = np.where(first, 0, 1)
    face_tets[sf, slot] = tidx[order_f]
    face_local[sf, slot] = lidx[order_f]

    pec_face = face_tag == 1
    pec_edge = np.zeros(edges.shape[0], dtype=bool)
    pec_tets = np.nonzero(pec_face[tet_faces])
    # edges of a PEC face: local face f of tet t contains local edges with both ends on the face
    for f in range(4):
        fl = set(LOCAL_FACES[f].tolist())
        le = [e for e in range(6) if set(LOCAL_EDGES[e].tolist()) <= fl]
        rows = pec_tets[0][pec_tets[1] == f]
        pec_edge[tet_edges[rows][:, le].ravel()] = True

    ne = edges.shape[0]
    edge_dof = -np.ones(ne, dtype=np.int64)
    keep_e = np.nonzero(~pec_edge)[0]
    edge_dof[keep_e] = np.arange(keep_e.size)
    if order == 1:
        tet_dofs = edge_dof[tet_edges]
        ndof = keep_e.size
        dof_kind = np.zeros(ndof, dtype=np.int64)
        dof_verts = np.concatenate([edges[keep_e], -np.ones((ndof, 1), dtype=np.int64)], axis=1)
    elif order == 2:
        nwe = keep_e.size
        grad_dof = np.where(edge_dof >= 0, edge_dof + nwe, -1)
        keep_f = np.nonzero(~pec_face)[0]
        face_dof = -np.ones(nf, dtype=np.int64)
        face_dof[keep_f] = 2 * nwe + 2 * np.arange(keep_f.size)
        fd = face_dof[tet_faces]  # [nt, 4]
        fa = np.where(fd >= 0, fd, -1)
        fb = np.where(fd >= 0, fd + 1, -1)
        face_part = np.stack([fa, fb], axis=2).reshape(nt, 8)
        tet_dofs = np.concatenate([edge_dof[tet_edges], grad_dof[tet_edges], face_part], axis=1)
        ndof = 2 * nwe + 2 * keep_f.size
        dof_kind = np.concatenate([np.zeros(nwe), np.ones(nwe),
                                   np.tile([2, 3], keep_f.size)]).astype(np.int64)
        ev_keep = np.concatenate([edges[keep_e], -np.ones((nwe, 1), dtype=np.int64)], axis=1)
        dof_verts = np.concatenate([ev_keep, ev_keep, np.repeat(faces[keep_f], 2, axis=0)], axis=0)
    else:
        raise ValueError("order must be 1 or 2")

    return Topology(order=order, nv=int(nv), tv=tv, edges=edges, tet_edges=tet_edges, faces=faces,
                    tet_faces=tet_faces, face_tag=face_tag, face_tets=face_tets,
                    face_local=face_local, pec_edge=pec_edge, tet_dofs=tet_dofs, ndof=int(ndof),
                    dof_kind=dof_kind, dof_verts=dof_verts)
