"""The second-order configuration at full size, checked with the oracle's operator.

487,080-tet chamber (48 x 45 grid), second-order edge elements (3,041,730
DOFs), 160 transmitters in 5 rings of 32, ORAS with 256 subdomains, mixed
path (complex FP32 factors and tensor-core sweeps inside the double-float
FGMRES) to rtol 1e-6, blocks of 32 columns, restart 30.  A direct oracle solve
of 3 M complex unknowns is out of reach on the host, so the fields are checked
against the oracle's own assembled operator and right-hand sides on a 64-column
subset: every column's true relative residual ||A u - b|| / ||b||, computed in
complex128 with the oracle's operator, must be within 5 % of rtol (the solver
tests its own residual in double-float), and S must be the oracle's receiver
map of the returned fields.
"""

import numpy as np
import pytest

import oracle as O
from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas
from tests._helpers import FREQ, key_perm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_second_order_160_columns_meet_rtol_with_oracle_operator():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi

    mesh = chamber_mesh(48, 45)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    ants = antenna_array([a for z in (0.06, 0.10, 0.14, 0.18, 0.22) for a in ring_antennas(32, z=z)])
    assert mesh.nt == 487080 and ants.shape[0] == 160
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag, order=2)
    assert M.ndof == 3041730
    rtol = 1e-6
    P = mwi.Problem(M, eps, FREQ, n_sub=256, precision=1, rtol=rtol, max_block=32, restart=30)
    S = P.forward_solve(ants, ants)
    info = P.info.as_dict()
    assert info["n_converged"] == 160 and info["resid_max"] <= rtol, info
    U = P.fields_host(0)
    kind, verts = M.dof_keys()
    P.close()
    M.close()
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 2)
    perm = key_perm(kind, verts, topo)
    cols = np.arange(0, 160, 160 // 64)[:64]  # 64 columns, every ring
    u = np.empty((topo.ndof, cols.size), dtype=np.complex128)
    u[perm] = U[:, cols]
    del U
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ).tocsr()
    tdof, tsgn = O.antenna_edges(mesh.xyz, topo, ants)
    b = O.build_rhs(topo.ndof, tdof[cols], tsgn[cols], ants[cols, 6] + 1j * ants[cols, 7], FREQ)
    r = np.linalg.norm(A @ u - b, axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 1.05 * rtol, r
    # S from the oracle's receiver map and the returned fields
    S_o = O.s_matrix(u, tdof, tsgn)
    assert np.abs(S_o - S[:, cols]).max() <= 1e-12 * np.abs(S_o).max()
