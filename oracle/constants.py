"""Physical constants (SI).  k0 = omega sqrt(mu0 eps0) = 2 pi f / c0 (Section 2)."""

import math

C0 = 299792458.0                 # speed of light in vacuum (m/s)
MU0 = 4.0e-7 * math.pi           # permeability of free space (H/m)


def k0_of(freq_hz):
    return 2.0 * math.pi * freq_hz / C0
