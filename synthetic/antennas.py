"""Antenna sets: edge-current dipoles given by a position, a direction and a current.

The paper's antennas are ceramic-loaded waveguides on 5 rings of 32 around the
chamber (Section 1); their geometry is not given, so each antenna here is a
point dipole that the solver attaches to a mesh edge.
"""

from dataclasses import dataclass

import numpy as np


@dataclass
class Antenna:
    pos: tuple
    dir: tuple = (0.0, 0.0, 1.0)
    current: complex = 1.0 + 0.0j


def cube_antennas(side=0.1):
    """Four +z dipoles at the centres of the four lateral faces of the cube."""
    h = 0.5 * side
    pts = [(0.0, h, h), (side, h, h), (h, 0.0, h), (h, side, h)]
    return [Antenna(pos=p) for p in pts]


def ring_antennas(n=32, radius=0.135, z=0.14):
    """n +z dipoles equally spaced on a ring (angle 2 pi k / n)."""
    out = []
    for k in range(n):
        a = 2.0 * np.pi * k / n
        out.append(Antenna(pos=(radius * np.cos(a), radius * np.sin(a), z)))
    return out


def antenna_array(ants):
    """Pack antennas as an [n, 8] float64 array: pos(3), dir(3), Re I, Im I."""
    a = np.zeros((len(ants), 8), dtype=np.float64)
    for i, t in enumerate(ants):
        a[i, 0:3] = t.pos
        a[i, 3:6] = t.dir
        a[i, 6] = complex(t.current).real
        a[i, 7] = complex(t.current).imag
    return a
