"""The antenna -> edge map of the forward solve without a GPU: the library's
grid search for the nearest vertex, through the host-only entry point
mwi_antenna_map_host, against the oracle's exhaustive search (antenna_edges).

* random positions inside and around the mesh (up to 30 % beyond its box),
  positions far outside it, positions on vertices, edge midpoints and hex
  centres of an unjittered cube (equidistant vertices: the lowest id wins),
  random directions: the same edge DOF and sign for every antenna;
* an antenna whose edge is a removed PEC edge, a zero direction and a
  non-finite position are refused (MWI_EINVAL).
"""

import numpy as np
import pytest

import oracle as O
from synthetic import chamber_mesh, cube_mesh
from tests._helpers import key_perm

mwi = pytest.importorskip("paper_1607_02573_gb300.mwi")


def _antennas(mesh, rng, n_random=150):
    lo, hi = mesh.xyz.min(0), mesh.xyz.max(0)
    ext = hi - lo
    pos = [lo - 0.3 * ext + 1.6 * ext * rng.random((n_random, 3)),
           lo + ext * np.array([[5.0, 0.5, 0.5], [-7.0, 3.0, -2.0], [0.5, 0.5, 40.0]]),
           mesh.xyz[rng.choice(mesh.nv, 20, replace=False)]]
    tet = np.asarray(mesh.tet)[rng.choice(len(mesh.tet), 20, replace=False)]
    pos.append(0.5 * (mesh.xyz[tet[:, 0]] + mesh.xyz[tet[:, 1]]))
    pos.append(mesh.xyz[tet].mean(axis=1))
    pos = np.concatenate(pos)
    d = rng.standard_normal(pos.shape)
    cur = rng.standard_normal((pos.shape[0], 2))
    return np.concatenate([pos, d, cur], axis=1)


def _oracle_one(mesh, topo, a):
    try:
        dof, sign = O.antenna_edges(mesh.xyz, topo, a[None])
        return int(dof[0]), float(sign[0])
    except ValueError:
        return None


@pytest.mark.parametrize("case,order", [("chamber", 1), ("chamber", 2), ("cube", 1), ("cube", 2)])
def test_antenna_map_matches_exhaustive_oracle(case, order):
    mesh = chamber_mesh(10, 9) if case == "chamber" else cube_mesh(5)
    if case == "cube":  # unjittered hexes: hex centres and midpoints give exact distance ties
        c = np.arange(4) * 0.02 + 0.01
        extra = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    else:
        extra = np.empty((0, 3))
    rng = np.random.default_rng(7 + order)
    ants = _antennas(mesh, rng)
    if extra.size:
        e = np.concatenate([extra, rng.standard_normal(extra.shape), np.ones((len(extra), 2))], axis=1)
        ants = np.concatenate([ants, e])
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    ref = [_oracle_one(mesh, topo, a) for a in ants]
    ok = np.array([r is not None for r in ref])
    assert ok.sum() >= 0.3 * len(ants)
    dof, sign, (kind, verts) = mwi.antenna_map_host(mesh, ants[ok], order)
    perm = key_perm(kind, verts, topo)
    want = np.array([r for r in ref if r is not None])
    assert np.array_equal(perm[dof], want[:, 0].astype(np.int64))
    assert np.array_equal(sign, want[:, 1])
    # every antenna the oracle puts on a removed PEC edge is refused
    for a in ants[~ok][:10]:
        with pytest.raises(mwi.MwiError, match="PEC"):
            mwi.antenna_map_host(mesh, a[None], order)


def test_bad_antennas_are_refused():
    mesh = cube_mesh(3)
    a = np.array([[0.05, 0.05, 0.05, 1.0, 0.0, 0.0, 1.0, 0.0]])
    mwi.antenna_map_host(mesh, a)
    for col, val in [(3, 0.0), (0, np.nan), (1, np.inf)]:
        b = a.copy()
        if col == 3:
            b[0, 3:6] = 0.0
        else:
            b[0, col] = val
        with pytest.raises(mwi.MwiError, match="MWI_EINVAL"):
            mwi.antenna_map_host(mesh, b)
