"""One forward solve on a synthetic chamber, for profiling under ncu and for
sizing runs.

python -m paper_1607_02573_gb300.profile_case NXY NZ N_SUB PRECISION [N_ANT ORDER RINGS MAX_BLOCK RESTART]

Defaults 30 28 32 1 32 1 1 64 50: 120,288 tets, 32 subdomains, mixed precision,
one ring of 32 antennas at z = 0.14 m, lowest order.  RINGS = 5 places rings at
z = 0.06, 0.10, 0.14, 0.18, 0.22 m (the 160-antenna layout).
"""

import os
import sys
import time


def main(argv):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np

    from paper_1607_02573_gb300 import mwi
    from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas

    defaults = [30, 28, 32, 1, 32, 1, 1, 64, 50]
    nxy, nz, n_sub, prec, n_ant, order, rings, max_block, restart = (list(map(int, argv)) +
                                                                     defaults[len(argv):])[:9]
    t0 = time.time()
    mesh = chamber_mesh(nxy, nz)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    zs = [0.14] if rings == 1 else [0.06, 0.10, 0.14, 0.18, 0.22]
    ants = []
    for z in zs:
        ants += ring_antennas(n_ant, z=z)
    ants = antenna_array(ants)
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag, order=order)
    t1 = time.time()
    P = mwi.Problem(M, eps, 1e9, n_sub=n_sub, precision=prec, rtol=1e-6, max_block=max_block, restart=restart)
    t2 = time.time()
    S = P.forward_solve(ants, ants, allow_notconv=True)
    t3 = time.time()
    info = P.info.as_dict()
    print(f"tets {mesh.nt} dof {M.ndof} order {order} columns {ants.shape[0]}")
    print(f"mesh {t1 - t0:.1f} s, assemble+decompose+factorise {t2 - t1:.1f} s, forward {t3 - t2:.2f} s "
          f"({ants.shape[0] / (t3 - t2):.1f} RHS-solves/s)")
    print("factor", P.factor_stats())
    print("oras_bytes_per_call", P.oras_traffic(min(32, ants.shape[0])))
    print("solve", info)
    print("reciprocity", float(np.linalg.norm(S - S.T) / np.linalg.norm(S)))
    P.close()
    M.close()


if __name__ == "__main__":
    main(sys.argv[1:])
