"""Global system A u_j = b_j (Eq. linsys) from the variational form (Eq. pbdirectvarf).

A = sum_t (K_t - k0^2 eps_t M_t) + i sum_{impedance faces f} beta_f B_f, with
K_t, M_t, B_f the element integrals of ``fem`` (mu_r = 1, the medium is
non-magnetic, Section 2), PEC DOFs removed, and beta_f = k0 sqrt(eps_t) for
the tet t owning the boundary face f (principal square root: Re > 0, Im < 0
for a lossy medium, so the +i beta term is the outgoing first-order
Silver-Mueller condition for the time factor exp(+i w t)).

Right-hand side of transmitter j: an edge-current dipole of current I0 on the
mesh edge k_j gives b_j = -i omega mu0 I0 s_j e_{k_j}, where s_j = +-1 says
whether the antenna direction agrees with the edge orientation.
"""

import numpy as np
import scipy.sparse as sp

from .constants import MU0, k0_of
from .fem import element_matrices, face_matrix


def impedance_faces(topo):
    """(tet, local face) of every impedance boundary face."""
    f = np.nonzero(topo.face_tag == 2)[0]
    return topo.face_tets[f, 0], topo.face_local[f, 0]


def _scatter_symmetric(dofs, vals, n):
    """Sum local matrices vals[e, i, j] into an n x n matrix at (dofs[e,i], dofs[e,j]).

    Only pairs with row <= col are summed; the lower triangle is the mirror,
    so the result is symmetric bit for bit.
    """
    nl = dofs.shape[1]
    r = np.repeat(dofs, nl, axis=1).ravel()
    c = np.tile(dofs, (1, nl)).ravel()
    v = vals.reshape(vals.shape[0], -1).ravel()
    keep = (r >= 0) & (c >= 0) & (r <= c)
    U = sp.coo_matrix((v[keep], (r[keep], c[keep])), shape=(n, n)).tocsr()
    U.sum_duplicates()
    return (U + sp.triu(U, k=1).T).tocsr()


def assemble_system(xyz, topo, eps, freq, K=None, M=None):
    """Return the complex symmetric CSR matrix A of Eq. linsys."""
    eps = np.asarray(eps, dtype=np.complex128)
    k0 = k0_of(freq)
    if K is None or M is None:
        K, M = element_matrices(xyz, topo)
    vol = K.astype(np.complex128) - (k0 * k0) * eps[:, None, None] * M
    ft, fl = impedance_faces(topo)
    B = face_matrix(xyz, topo, ft, fl)
    beta = k0 * np.sqrt(eps[ft])
    bnd = 1j * beta[:, None, None] * B
    dofs = np.concatenate([topo.tet_dofs, topo.tet_dofs[ft]], axis=0)
    vals = np.concatenate([vol, bnd], axis=0)
    return _scatter_symmetric(dofs, vals, topo.ndof)


def antenna_edges(xyz, topo, antennas):
    """Map antennas [n, 8] (pos, dir, Re I, Im I) to (edge DOF, sign).

    The antenna edge starts at the mesh vertex nearest to pos (lowest vertex
    id on ties) and is, among the edges at that vertex, the one best aligned
    with dir (largest cosine; lowest global edge id on ties).  Raises if that
    edge is a removed PEC edge.
    """
    antennas = np.asarray(antennas, dtype=np.float64).reshape(-1, 8)
    dofs = np.empty(antennas.shape[0], dtype=np.int64)
    signs = np.empty(antennas.shape[0], dtype=np.float64)
    edge_dof = -np.ones(topo.edges.shape[0], dtype=np.int64)
    keep = np.nonzero(~topo.pec_edge)[0]
    edge_dof[keep] = np.arange(keep.size)
    for a, row in enumerate(antennas):
        pos, d = row[0:3], row[3:6]
        v = int(np.argmin(np.sum((xyz - pos) ** 2, axis=1)))
        inc = np.nonzero((topo.edges[:, 0] == v) | (topo.edges[:, 1] == v))[0]
        other = np.where(topo.edges[inc, 0] == v, topo.edges[inc, 1], topo.edges[inc, 0])
        vec = xyz[other] - xyz[v]
        cos = (vec @ d) / (np.linalg.norm(vec, axis=1) * np.linalg.norm(d))
        best = inc[np.argmax(cos)]  # inc is sorted, so ties go to the lowest edge id
        if edge_dof[best] < 0:
            raise ValueError(f"antenna {a} falls on a PEC edge")
        t = xyz[topo.edges[best, 1]] - xyz[topo.edges[best, 0]]
        dofs[a] = edge_dof[best]
        signs[a] = 1.0 if float(t @ d) > 0.0 else -1.0
    return dofs, signs


def build_rhs(ndof, dofs, signs, currents, freq):
    """b_j = -i omega mu0 I_j s_j e_{k_j}, columns j = 0..m-1."""
    omega = 2.0 * np.pi * freq
    b = np.zeros((ndof, len(dofs)), dtype=np.complex128)
    for j, (k, s, I) in enumerate(zip(dofs, signs, currents)):
        b[k, j] = -1j * omega * MU0 * I * s
    return b
