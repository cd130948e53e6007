"""One-level ORAS preconditioner and flexible GMRES (Section 3), plain CPU form.

Decomposition (Section 3):
* non-overlapping partition T_i of the tets by recursive coordinate bisection
  of tet centroids (the paper uses a graph partitioner; any partition is
  admissible).  At each step the tets are sorted by (centroid[axis], tet id)
  along the axis of largest centroid extent (lowest axis on ties) and split
  at floor(|T| p_left / p) with p_left = p // 2;
* overlap: T_i^d = T_i^{d-1} plus every tet adjacent to it, where adjacent
  means sharing a vertex;
* P1 partition of unity (Eq. chi): chi~_i = 1 at the nodes of T_i^0 and 0 at
  the other nodes of T_i^delta; chi_i = chi~_i / sum_j chi~_j;
* edge partition of unity: D_i[e] = chi_i at the midpoint of edge e (face
  DOFs of order 2: at the face centroid), so sum_i R_i^T D_i R_i = I
  (Eq. algebPartUnity);
* local operator B_i: the form of Eq. pbdirectvarf restricted to T_i^delta,
  plus the impedance condition i k int (E x n).(v x n) on the faces of
  T_i^delta interior to the domain, k = k0 sqrt(eps_t) of the tet of
  T_i^delta owning the face.

ORAS (Eq. ORAS):  M^{-1} r = sum_i R_i^T D_i B_i^{-1} R_i r, each B_i^{-1} by
sparse LU.  Two-level variant (Section 7): a coarse Whitney space on a coarser
mesh, Galerkin coarse operator, deflated combination with ORAS (CoarseSpace).  FGMRES: right-preconditioned flexible GMRES (restarted, x0 = 0,
modified Gram-Schmidt Arnoldi, Givens rotations), stopped on the
unpreconditioned relative residual (Section 6).
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assemble import _scatter_symmetric
from .constants import k0_of
from .fem import element_matrices, face_matrix


def rcb_partition(xyz, tet, nparts):
    P = xyz[np.asarray(tet)]
    c = (((P[:, 0] + P[:, 1]) + P[:, 2]) + P[:, 3]) / 4.0
    part = np.zeros(c.shape[0], dtype=np.int64)

    def rec(ids, p, first):
        if p == 1:
            part[ids] = first
            return
        cc = c[ids]
        ext = cc.max(axis=0) - cc.min(axis=0)
        ax = int(np.argmax(ext))
        order = np.lexsort((ids, cc[:, ax]))
        ids = ids[order]
        pl = p // 2
        cut = (ids.size * pl) // p
        rec(ids[:cut], pl, first)
        rec(ids[cut:], p - pl, first + pl)

    rec(np.arange(c.shape[0]), int(nparts), 0)
    return part


def grow_overlap(tet, in_sub, delta):
    """T^d: add every tet sharing a vertex with T^{d-1}, delta times."""
    tet = np.asarray(tet)
    sub = in_sub.copy()
    nv = int(tet.max()) + 1
    for _ in range(delta):
        vm = np.zeros(nv, dtype=bool)
        vm[tet[sub].ravel()] = True
        sub = vm[tet].any(axis=1)
    return sub


class Decomposition:
    def __init__(self, xyz, tet, topo, part, delta=1):
        self.nsub = int(part.max()) + 1
        self.part = part
        tet = np.asarray(tet)
        nv = xyz.shape[0]
        self.T0 = [part == i for i in range(self.nsub)]
        self.Td = [grow_overlap(tet, m, delta) for m in self.T0]
        chit = np.zeros((self.nsub, nv))
        for i in range(self.nsub):
            chit[i, np.unique(tet[self.T0[i]])] = 1.0
        chi = chit / chit.sum(axis=0, keepdims=True)
        self.chi = chi
        self.R, self.D = [], []
        for i in range(self.nsub):
            d = topo.tet_dofs[self.Td[i]].ravel()
            dofs = np.unique(d[d >= 0])
            self.R.append(dofs)
            vv = topo.dof_verts[dofs]
            cnt = (vv >= 0).sum(axis=1)
            vals = np.where(vv >= 0, chi[i][np.maximum(vv, 0)], 0.0).sum(axis=1) / cnt
            self.D.append(vals)


def local_matrices(xyz, topo, dec, eps, freq, K=None, M=None):
    """B_i for every subdomain, in the local numbering given by dec.R[i]."""
    eps = np.asarray(eps, dtype=np.complex128)
    k0 = k0_of(freq)
    if K is None or M is None:
        K, M = element_matrices(xyz, topo)
    vol = K.astype(np.complex128) - (k0 * k0) * eps[:, None, None] * M
    out = []
    for i in range(dec.nsub):
        inside = dec.Td[i]
        tets = np.nonzero(inside)[0]
        # faces of T_i^delta on its boundary: one tet of the face inside, the other outside or absent
        ft_all, fl_all, kind = [], [], []
        for s in range(2):
            t = topo.face_tets[:, s]
            o = topo.face_tets[:, 1 - s]
            ok = (t >= 0) & inside[np.maximum(t, 0)]
            other_out = (o < 0) | ~inside[np.maximum(o, 0)]
            sel = np.nonzero(ok & other_out)[0]
            ft_all.append(t[sel])
            fl_all.append(topo.face_local[sel, s])
            kind.append(topo.face_tag[sel])
        ft = np.concatenate(ft_all)
        fl = np.concatenate(fl_all)
        fk = np.concatenate(kind)
        use = fk != 1  # PEC faces carry no term (their DOFs are removed)
        ft, fl = ft[use], fl[use]
        B = face_matrix(xyz, topo, ft, fl)
        kb = k0 * np.sqrt(eps[ft])
        g2l = -np.ones(topo.ndof + 1, dtype=np.int64)
        g2l[dec.R[i]] = np.arange(dec.R[i].size)
        dl_t = g2l[topo.tet_dofs[tets]]
        dl_f = g2l[topo.tet_dofs[ft]]
        dofs = np.concatenate([dl_t, dl_f], axis=0)
        vals = np.concatenate([vol[tets], 1j * kb[:, None, None] * B], axis=0)
        out.append(_scatter_symmetric(dofs, vals, dec.R[i].size))
    return out


class ORAS:
    def __init__(self, dec, Bs):
        self.dec = dec
        self.lus = [spla.splu(B.tocsc(), permc_spec="MMD_AT_PLUS_A") for B in Bs]

    def apply(self, r):
        r = np.asarray(r, dtype=np.complex128)
        z = np.zeros_like(r)
        for i, lu in enumerate(self.lus):
            Ri = self.dec.R[i]
            yi = lu.solve(np.ascontiguousarray(r[Ri]))
            Di = self.dec.D[i]
            z[Ri] += Di.reshape((-1,) + (1,) * (r.ndim - 1)) * yi
        return z


def fgmres(A, b, precond, rtol=1e-8, restart=50, maxiter=1000):
    """Right-preconditioned flexible GMRES for one column (Saad, Alg. 9.6)."""
    b = np.asarray(b, dtype=np.complex128)
    n = b.size
    x = np.zeros(n, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    r = b.copy()
    beta = np.linalg.norm(r)
    hist.append(beta / bnorm)
    while it < maxiter and beta / bnorm > rtol:
        V = np.zeros((restart + 1, n), dtype=np.complex128)
        Z = np.zeros((restart, n), dtype=np.complex128)
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(restart):
            Z[k] = precond(V[k])
            w = A @ Z[k]
            for i in range(k + 1):
                H[i, k] = np.vdot(V[i], w)
                w = w - H[i, k] * V[i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0.0:
                V[k + 1] = w / H[k + 1, k]
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -np.conj(sn[i]) * H[i, k] + np.conj(cs[i]) * H[i + 1, k]
                H[i, k] = t
            a, bb = H[k, k], H[k + 1, k]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            # unitary rotation [c s; -conj(s) conj(c)] mapping [a; b] to [den; 0]
            cs[k] = np.conj(a) / den if den != 0 else 1.0
            sn[k] = np.conj(bb) / den if den != 0 else 0.0
            H[k, k] = cs[k] * a + sn[k] * bb
            H[k + 1, k] = 0.0
            g[k + 1] = -np.conj(sn[k]) * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            k_done = k + 1
            hist.append(abs(g[k + 1]) / bnorm)
            if abs(g[k + 1]) / bnorm <= rtol or it >= maxiter:
                break
        y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + Z[:k_done].T @ y
        r = b - A @ x
        beta = np.linalg.norm(r)
        hist[-1] = beta / bnorm
    return x, it, hist


def solve_oras(A, B, oras, rtol=1e-10, restart=50, maxiter=1000):
    """FGMRES + ORAS for every column of B; returns U, iteration counts."""
    B = np.asarray(B, dtype=np.complex128)
    U = np.zeros_like(B)
    its = []
    for j in range(B.shape[1]):
        U[:, j], it, _ = fgmres(A, B[:, j], oras.apply, rtol=rtol, restart=restart, maxiter=maxiter)
        its.append(it)
    return U, its


class CoarseSpace:
    """Two-level ORAS with a geometric coarse space (Section 7 names a
    two-level preconditioner with a coarse space as what a one-level method
    needs to scale to thousands of subdomains).

    Coarse space: lowest-order Whitney elements on a coarser tetrahedral mesh
    of the same domain.  The prolongation maps coarse DOFs to fine edge DOFs by
    the fine edge's tangential integral of the coarse field, midpoint rule:
      P[e, E] = N_E(m_e) . (x_hi(e) - x_lo(e)),
    N_E evaluated in the coarse tet that holds the midpoint m_e, found by
    brute force over all coarse tets: the lowest-numbered tet whose smallest
    barycentric coordinate of m_e is >= -1e-12; for a midpoint in no tet
    (outside the coarse mesh), the lowest-numbered tet whose smallest
    barycentric coordinate is within 1e-12 of the largest over all tets (the
    affine extension of the least-outside tet's basis).  Ties go to the lowest
    tet number, so that rounding and search order cannot change the choice:
    N_E's normal component jumps across coarse faces, and exact ties are
    common on structured coarse meshes.  Coarse operator A_c = P^T A P
    (Galerkin; A is complex symmetric, so P^T).  Deflated two-level
    preconditioner:
      M_2 r = M_ORAS (r - A Q r) + Q r,   Q = P A_c^{-1} P^T.
    """

    def __init__(self, fine_xyz, fine_topo, coarse_xyz, coarse_topo, A, oras):
        from .fem import bary_gradients
        from .topology import LOCAL_EDGES

        ctv = coarse_topo.tv
        P4 = coarse_xyz[ctv]
        G, _ = bary_gradients(P4)
        cen = P4.mean(axis=1)
        e = fine_topo.edges
        fdof = np.full(e.shape[0], -1, dtype=np.int64)
        fdof[fine_topo.tet_edges.ravel()] = fine_topo.tet_dofs[:, :6].ravel()
        live = np.nonzero(fdof >= 0)[0]
        mid = 0.5 * (fine_xyz[e[live, 0]] + fine_xyz[e[live, 1]])
        tang = fine_xyz[e[live, 1]] - fine_xyz[e[live, 0]]
        t = np.empty(live.size, dtype=np.int64)
        L = np.empty((live.size, 4))
        for a in range(0, live.size, 64):
            b = min(live.size, a + 64)
            # barycentric coordinates of every midpoint in every coarse tet:
            # lambda_q is affine with gradient G_q and equals 1/4 at the centroid
            lam = np.einsum("tqd,ntd->ntq", G, mid[a:b, None, :] - cen[None, :, :]) + 0.25
            mins = lam.min(axis=2)
            inside = mins >= -1e-12
            near = mins >= mins.max(axis=1, keepdims=True) - 1e-12
            pick = np.where(inside.any(axis=1), inside.argmax(axis=1), near.argmax(axis=1))
            t[a:b] = pick
            L[a:b] = lam[np.arange(b - a), pick]
        self.located = (fdof[live], t)  # (fine DOF, coarse tet) of every live fine Whitney edge
        rows, cols, vals = [], [], []
        for j, (a, b) in enumerate(LOCAL_EDGES):
            N = L[:, a, None] * G[t, b] - L[:, b, None] * G[t, a]
            cd = coarse_topo.tet_dofs[t, j]
            ok = cd >= 0
            rows.append(fdof[live][ok])
            cols.append(cd[ok])
            vals.append(np.einsum("nd,nd->n", N[ok], tang[ok]))
        self.P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(fine_topo.ndof, coarse_topo.ndof)).tocsr()
        self.A = A
        self.oras = oras
        self.Ac = (self.P.T @ A @ self.P).tocsc()
        self.lu = spla.splu(self.Ac, permc_spec="MMD_AT_PLUS_A")

    def coarse_correction(self, r):
        """Q r = P A_c^{-1} P^T r."""
        return self.P @ self.lu.solve(np.asarray(self.P.T @ r, dtype=np.complex128))

    def apply(self, r):
        """Deflated two-level preconditioner M_ORAS (r - A Q r) + Q r."""
        q = self.coarse_correction(r)
        return self.oras.apply(r - self.A @ q) + q
