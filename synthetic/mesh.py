"""Seeded structured-to-unstructured tetrahedral meshes.

Every hexahedron of an axis-aligned grid is split into the six Kuhn tetrahedra
that share its main diagonal (the split is translation invariant, so the mesh
is conforming).  Interior vertices may be jittered, and vertex ids, tet ids and
the vertex order inside each tet are randomly permuted so that a consumer of
the mesh cannot rely on any grid ordering.

Boundary tags per tet face (face k is the face opposite local vertex k):
0 = interior, 1 = perfectly conducting wall (PEC), 2 = impedance boundary.
"""

from dataclasses import dataclass
from itertools import permutations

import numpy as np

TAG_INTERIOR = 0
TAG_PEC = 1
TAG_IMPEDANCE = 2


@dataclass
class Mesh:
    xyz: np.ndarray        # [nv, 3] float64 vertex coordinates (m)
    tet: np.ndarray        # [nt, 4] int32 vertex ids
    bface_tag: np.ndarray  # [nt, 4] int32, tag of the face opposite local vertex k
    h: float               # grid spacing (m)
    name: str = ""

    @property
    def nv(self):
        return self.xyz.shape[0]

    @property
    def nt(self):
        return self.tet.shape[0]


_KUHN_PERMS = list(permutations(range(3)))


def _signed_volumes(xyz, tet):
    p0 = xyz[tet[:, 0]]
    e1 = xyz[tet[:, 1]] - p0
    e2 = xyz[tet[:, 2]] - p0
    e3 = xyz[tet[:, 3]] - p0
    return np.einsum("ij,ij->i", e1, np.cross(e2, e3)) / 6.0


def kuhn_box_mesh(n, lo, hi, keep_hex=None, impedance="all", jitter=0.0,
                  seed_jitter=7, seed_perm=11, permute=True, name=""):
    """Kuhn-split mesh of the box [lo, hi] with n = (nx, ny, nz) hexes per axis.

    keep_hex(centres[nh, 3]) -> bool mask selects the hexes kept (default all).
    impedance: "all" tags every boundary face as impedance; "top" tags only the
    faces on the plane z = hi[2] as impedance and every other boundary face PEC.
    jitter: interior vertices move by U(-jitter*h, jitter*h) per axis.
    """
    nx, ny, nz = (int(v) for v in n)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    ext = hi - lo
    hx = ext / np.array([nx, ny, nz], dtype=np.float64)

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    I, J, K = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    I = I.ravel(); J = J.ravel(); K = K.ravel()
    if keep_hex is not None:
        centres = lo + (np.stack([I, J, K], axis=1) + 0.5) * hx
        mask = np.asarray(keep_hex(centres), dtype=bool)
        I = I[mask]; J = J[mask]; K = K[mask]

    tets = []
    for perm in _KUHN_PERMS:
        step = np.zeros(3, dtype=np.int64)
        corners = [vid(I, J, K)]
        for ax in perm:
            step[ax] += 1
            corners.append(vid(I + step[0], J + step[1], K + step[2]))
        tets.append(np.stack(corners, axis=1))
    tet = np.concatenate(tets, axis=0).astype(np.int64)

    # grid coordinates of every grid vertex (top plane exactly at hi)
    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    gidx = np.stack([gi.ravel(order="F"), gj.ravel(order="F"), gk.ravel(order="F")], axis=1)
    # order="F" so that row r corresponds to vid = i + (nx+1)*(j + (ny+1)*k)
    gxyz = lo + ext * (gidx / np.array([nx, ny, nz], dtype=np.float64))

    # boundary faces: faces used by exactly one tet
    nt = tet.shape[0]
    face_local = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])  # face opposite vertex k
    fv = np.sort(tet[:, face_local], axis=2)  # [nt, 4, 3]
    ng = (nx + 1) * (ny + 1) * (nz + 1)
    keys = (fv[:, :, 0] * ng + fv[:, :, 1]) * ng + fv[:, :, 2]
    _, inv, cnt = np.unique(keys.ravel(), return_inverse=True, return_counts=True)
    is_bnd = (cnt[inv] == 1).reshape(nt, 4)
    tag = np.zeros((nt, 4), dtype=np.int32)
    if impedance == "all":
        tag[is_bnd] = TAG_IMPEDANCE
    elif impedance == "top":
        ktop = gidx[fv, 2] == nz  # [nt, 4, 3]
        top = ktop.all(axis=2)
        tag[is_bnd & top] = TAG_IMPEDANCE
        tag[is_bnd & ~top] = TAG_PEC
    else:
        raise ValueError("impedance must be 'all' or 'top'")

    # compact the used vertices
    used = np.unique(tet)
    remap = -np.ones(ng, dtype=np.int64)
    remap[used] = np.arange(used.size)
    xyz = gxyz[used].copy()
    tet = remap[tet]
    bnd_vert = np.zeros(used.size, dtype=bool)
    bnd_vert[remap[fv[is_bnd].ravel()]] = True

    vol0 = _signed_volumes(xyz, tet)
    if jitter > 0.0:
        rng = np.random.default_rng(seed_jitter)
        h = float(hx.min())
        d = rng.uniform(-jitter * h, jitter * h, size=(ng, 3))[used]
        d[bnd_vert] = 0.0
        xyz = xyz + d
        vol = _signed_volumes(xyz, tet)
        if not np.all(np.sign(vol) == np.sign(vol0)) or np.abs(vol).min() <= 0.0:
            raise RuntimeError("jitter inverted a tetrahedron")

    if permute:
        rng = np.random.default_rng(seed_perm)
        nv = xyz.shape[0]
        vperm = rng.permutation(nv)          # new id of old vertex v
        tperm = rng.permutation(tet.shape[0])  # old tet at new position
        local = np.argsort(rng.random((tet.shape[0], 4)), axis=1)
        xyz_new = np.empty_like(xyz)
        xyz_new[vperm] = xyz
        tet = vperm[tet]
        tet = np.take_along_axis(tet, local, axis=1)[tperm]
        tag = np.take_along_axis(tag, local, axis=1)[tperm]
        xyz = xyz_new

    return Mesh(xyz=np.ascontiguousarray(xyz, dtype=np.float64),
                tet=np.ascontiguousarray(tet, dtype=np.int32),
                bface_tag=np.ascontiguousarray(tag, dtype=np.int32),
                h=float(hx.min()), name=name)


def cube_mesh(n=8, side=0.1, jitter=0.0, permute=True):
    """Cube [0, side]^3 with n^3 hexes (6 n^3 tets), impedance on all faces."""
    return kuhn_box_mesh((n, n, n), (0.0, 0.0, 0.0), (side, side, side), impedance="all",
                         jitter=jitter, permute=permute, name=f"cube{n}")


CHAMBER_RADIUS = 0.15
CHAMBER_HEIGHT = 0.28


def chamber_mesh(nxy=45, nz=42, radius=CHAMBER_RADIUS, height=CHAMBER_HEIGHT, jitter=0.15, permute=True):
    """Cylindrical chamber (axis x = y = 0, 0 <= z <= height).

    Hexes of a (nxy, nxy, nz) grid over [-r, r]^2 x [0, height] are kept when
    their centre lies inside the cylinder (staircase wall).  The lateral wall
    and bottom are PEC; the top plane z = height is an impedance boundary.
    """
    def keep(c):
        return c[:, 0] ** 2 + c[:, 1] ** 2 < radius ** 2

    return kuhn_box_mesh((nxy, nxy, nz), (-radius, -radius, 0.0), (radius, radius, height),
                         keep_hex=keep, impedance="top", jitter=jitter, permute=permute,
                         name=f"chamber{nxy}x{nxy}x{nz}")
