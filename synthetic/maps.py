"""Seeded relative-permittivity maps, one complex value per tetrahedron.

Values follow the time factor exp(+i w t) of Section 2, so lossy media have a
negative imaginary part: matching gel 44 - 20i (Section 4), blood 68 - 44i
(Section 6.2).  Each map is sampled at tet centroids.
"""

import numpy as np

EPS_GEL = 44.0 - 20.0j          # matching medium (Section 4)
EPS_HEAD = 45.0 - 18.0j         # head-sized ellipsoid of the chamber workloads
EPS_BLOOD_LIKE = 60.0 - 25.0j   # high-contrast inclusion (haemorrhage-like)
EPS_LOW = 38.0 - 15.0j          # low-contrast inclusion (ischaemia-like)

HEAD_CENTRE = np.array([0.0, 0.0, 0.14])
HEAD_AXES = np.array([0.09, 0.07, 0.10])
INCLUSION_RADIUS = 0.015


def tet_centroids(xyz, tet):
    return xyz[tet].mean(axis=1)


def cube_eps(xyz, tet, seed=1, side=0.1):
    """Gel background plus one sphere (r = 0.02 m) of 60 - 25i.

    The centre is drawn uniformly in [0.3, 0.7]^3 * side with the given seed.
    """
    rng = np.random.default_rng(seed)
    centre = rng.uniform(0.3 * side, 0.7 * side, size=3)
    c = tet_centroids(xyz, tet)
    eps = np.full(tet.shape[0], EPS_GEL, dtype=np.complex128)
    eps[np.sum((c - centre) ** 2, axis=1) < 0.02 ** 2] = EPS_BLOOD_LIKE
    return eps


def _draw_inside_shrunk_ellipsoid(rng, r):
    axes = HEAD_AXES - r
    while True:
        p = rng.uniform(-1.0, 1.0, size=3)
        if np.sum(p * p) <= 1.0:
            return HEAD_CENTRE + p * axes


def _head(c):
    return np.sum(((c - HEAD_CENTRE) / HEAD_AXES) ** 2, axis=1) < 1.0


def chamber_eps(xyz, tet, seed=2, inclusions=(EPS_BLOOD_LIKE,)):
    """Gel, head ellipsoid (45 - 18i) and seeded spherical inclusions inside it."""
    rng = np.random.default_rng(seed)
    c = tet_centroids(xyz, tet)
    eps = np.full(tet.shape[0], EPS_GEL, dtype=np.complex128)
    eps[_head(c)] = EPS_HEAD
    for value in inclusions:
        centre = _draw_inside_shrunk_ellipsoid(rng, INCLUSION_RADIUS)
        eps[np.sum((c - centre) ** 2, axis=1) < INCLUSION_RADIUS ** 2] = value
    return eps


def chamber_target_eps(xyz, tet, seed=3):
    """Inversion target: head ellipsoid with two inclusions (60 - 25i, 38 - 15i)."""
    return chamber_eps(xyz, tet, seed=seed, inclusions=(EPS_BLOOD_LIKE, EPS_LOW))
