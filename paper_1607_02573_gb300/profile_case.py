"""One forward solve on a synthetic chamber, for profiling under ncu.

python -m paper_1607_02573_gb300.profile_case NXY NZ N_SUB PRECISION [N_ANT]
(defaults 30 28 32 1 32: 120,288 tets, 32 subdomains, mixed precision, 32 antennas).
"""

import os
import sys


def main(argv):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1607_02573_gb300 import mwi
    from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas

    nxy, nz, n_sub, prec, n_ant = (list(map(int, argv)) + [30, 28, 32, 1, 32][len(argv):])[:5]
    mesh = chamber_mesh(nxy, nz)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    ants = antenna_array(ring_antennas(n_ant))
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = mwi.Problem(M, eps, 1e9, n_sub=n_sub, precision=prec, rtol=1e-6)
    P.forward_solve(ants, ants)
    print(mesh.nt, M.ndof, P.factor_stats(), P.info.as_dict())
    P.close()
    M.close()


if __name__ == "__main__":
    main(sys.argv[1:])
