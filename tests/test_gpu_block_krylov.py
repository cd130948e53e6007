"""GPU parity of the true block FGMRES (one Krylov space shared by the
columns of a block, the block methods of Section 7) through the C ABI.

* after a fixed number of block steps the iterate equals the oracle's block
  FGMRES iterate with the same ORAS preconditioner (both are the least-residual
  element of the same block space): <= 1e-8 relative in FP64;
* solved to tolerance, fields and S match the direct oracle solution: FP64 path
  rtol 1e-12 -> <= 1e-8, FP32 ORAS preconditioner rtol 1e-9 -> <= 1e-6, also
  when the transmitters are split over several blocks;
* it needs no more steps than the pseudo-block FGMRES (each column's own space
  is inside the block space);
* a repeated transmitter makes the block of right-hand sides rank deficient:
  the Cholesky QR deflates the copy and both columns still get the solution.
"""

import numpy as np
import pytest

import oracle as O
from oracle import block_gmres as bg
from oracle import dd
from tests._helpers import FREQ, chamber_case, col_rel_err, key_perm, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    return mwi


@pytest.fixture(scope="module")
def chamber(lib):
    mesh, eps, tx, rx = chamber_case(12, 11, n_ant=6)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    kind, verts = M.dof_keys()
    perm = key_perm(kind, verts, topo)
    ref = O.forward(mesh.xyz, topo, eps, FREQ, tx, rx)
    yield mesh, eps, tx, rx, M, topo, perm, ref
    M.close()


def test_fixed_steps_match_oracle_block_fgmres(lib, chamber):
    mesh, eps, tx, rx, M, topo, perm, ref = chamber
    part = dd.rcb_partition(mesh.xyz, mesh.tet, 4)
    steps = 3
    P = lib.Problem(M, eps, FREQ, n_sub=4, part=part, precision=0, block_krylov=1, rtol=1e-15,
                    max_iter=steps, restart=10)
    P.forward_solve(tx, rx, allow_notconv=True)
    assert P.info.iters_max == steps
    U = P.fields_host(0)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    oras = dd.ORAS(dec, dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ))
    X, _, k = bg.block_fgmres(ref["A"].tocsr(), ref["b"], oras.apply, steps=steps)
    assert k == steps
    assert rel_err(U, X[perm]) <= 1e-8
    P.close()


@pytest.mark.parametrize("precision,rtol,tol,max_block", [(0, 1e-12, 1e-8, 64), (1, 1e-9, 1e-6, 64),
                                                          (1, 1e-9, 1e-6, 4)])
def test_solution_matches_direct_oracle(lib, chamber, precision, rtol, tol, max_block):
    mesh, eps, tx, rx, M, topo, perm, ref = chamber
    P = lib.Problem(M, eps, FREQ, n_sub=6, precision=precision, block_krylov=1, rtol=rtol, max_iter=300,
                    max_block=max_block)
    S = P.forward_solve(tx, rx)
    assert P.info.n_converged == tx.shape[0]
    assert P.info.resid_max <= rtol
    U = P.fields_host(0)
    assert col_rel_err(U, ref["U"][perm]).max() <= tol
    assert rel_err(S, ref["S"]) <= tol
    P.close()


def test_no_more_steps_than_pseudo_block(lib, chamber):
    mesh, eps, tx, rx, M, topo, perm, ref = chamber
    its = {}
    for block in (0, 1):
        P = lib.Problem(M, eps, FREQ, n_sub=6, precision=0, block_krylov=block, rtol=1e-10, max_iter=300)
        P.forward_solve(tx, rx)
        its[block] = P.info.iters_max
        P.close()
    assert its[1] <= its[0], its


def test_repeated_transmitter_is_deflated(lib, chamber):
    mesh, eps, tx, rx, M, topo, perm, ref = chamber
    tx2 = np.vstack([tx[:3], tx[1:2]])
    P = lib.Problem(M, eps, FREQ, n_sub=6, precision=0, block_krylov=1, rtol=1e-11, max_iter=300)
    S = P.forward_solve(tx2, rx)
    assert P.info.n_converged == 4
    U = P.fields_host(0)
    Uo = ref["U"][perm][:, [0, 1, 2, 1]]
    assert col_rel_err(U, Uo).max() <= 1e-7
    assert rel_err(S, ref["S"][:, [0, 1, 2, 1]]) <= 1e-7  # [receiver, transmitter]
    P.close()


@pytest.mark.parametrize("precision,rtol,tol", [(0, 1e-11, 1e-8), (1, 1e-9, 1e-6)])
def test_restarted_block_solver(lib, chamber, precision, rtol, tol):
    """Restart length 2: many block cycles, each from the true residual with a
    fresh block basis; the result still matches the direct oracle."""
    mesh, eps, tx, rx, M, topo, perm, ref = chamber
    P = lib.Problem(M, eps, FREQ, n_sub=6, precision=precision, block_krylov=1, restart=2, rtol=rtol, max_iter=400)
    S = P.forward_solve(tx, rx)
    assert P.info.n_converged == tx.shape[0]
    assert P.info.iters_max > 2
    assert col_rel_err(P.fields_host(0), ref["U"][perm]).max() <= tol
    assert rel_err(S, ref["S"]) <= tol
    P.close()
