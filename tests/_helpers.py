"""Shared test plumbing: DOF-key matching between the library and the oracle,
workload builders and tolerances.  No method arithmetic lives here."""

import numpy as np

import oracle as O
from synthetic import (antenna_array, chamber_eps, chamber_mesh, cube_antennas, cube_eps, cube_mesh,
                       ring_antennas)

FREQ = 1e9


def key_perm(lib_kind, lib_verts, topo):
    """perm[i] = oracle DOF index of library DOF i (matched on (kind, vertices))."""
    n = topo.ndof
    assert lib_kind.shape[0] == n
    nv = topo.nv + 1

    def keys(kind, verts):
        v = verts.astype(np.int64) + 1  # -1 -> 0
        return ((kind.astype(np.int64) * nv + v[:, 0]) * nv + v[:, 1]) * nv + v[:, 2]

    kl = keys(lib_kind, lib_verts)
    ko = keys(topo.dof_kind, topo.dof_verts)
    ol = np.argsort(kl)
    oo = np.argsort(ko)
    assert np.array_equal(kl[ol], ko[oo]), "library and oracle DOF sets differ"
    perm = np.empty(n, dtype=np.int64)
    perm[ol] = oo
    return perm


def cube_case(n=8, order=1):
    mesh = cube_mesh(n)
    eps = cube_eps(mesh.xyz, mesh.tet)
    ants = antenna_array(cube_antennas())
    return mesh, eps, ants, ants


def chamber_case(nxy=16, nz=15, order=1, n_ant=8, radius=0.1):
    mesh = chamber_mesh(nxy, nz)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    ants = antenna_array(ring_antennas(n_ant, radius=radius))
    return mesh, eps, ants, ants


def rel_err(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def col_rel_err(a, b):
    return np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)


def unpack_pairs(nl):
    """(i, j), i <= j, of every packed local pair index i nl - i (i-1)/2 + j - i
    of the library's element contributions."""
    return {i * nl - i * (i - 1) // 2 + (j - i): (i, j) for i in range(nl) for j in range(i, nl)}
