"""GPU parity of Krylov recycling across nearby systems (the recycling named in
Section 7; the previous L-BFGS step's solution block spans the recycled space)
through the C ABI.

* the recycled initial guess equals the oracle's least-residual element of the
  span of the previous solutions (FP32 normal equations: <= 1e-3 relative, its
  residual norms to 1e-3), checked with a loose rtol that the guess already
  meets (no Krylov step taken);
* with recycling, the forward fields, S, the misfit and the gradient of the
  next, perturbed system still match the direct oracle solution (FP64 path
  rtol 1e-12 -> <= 1e-8; mixed path rtol 1e-9 -> <= 1e-6), in fewer
  iterations than the same solve started from zero;
* solving the same system again starts from (nearly) its solution.
"""

import numpy as np
import pytest

import oracle as O
from oracle import block_gmres as bg
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
    rng = np.random.default_rng(21)
    eps2 = eps * (1 + 0.03 * rng.uniform(-1, 1, mesh.nt))
    ref2 = O.forward(mesh.xyz, topo, eps2, FREQ, tx, rx)
    yield mesh, eps, eps2, tx, rx, M, topo, perm, ref2
    M.close()


def test_recycled_guess_matches_oracle(lib, chamber):
    mesh, eps, eps2, tx, rx, M, topo, perm, ref2 = chamber
    P = lib.Problem(M, eps, FREQ, n_sub=6, precision=0, recycle=1, rtol=0.9, max_iter=50)
    P.forward_solve(tx, rx)
    X1 = P.fields_host(0)
    P.update_eps(eps2)
    P.forward_solve(tx, rx)
    assert P.info.iters_max == 0
    X2 = P.fields_host(0)
    inv = np.argsort(perm)
    A2 = ref2["A"].tocsr()
    x0 = bg.recycled_initial_guess(A2, ref2["b"], X1[inv])
    # FP32 normal equations: the guess to ~kappa(C)^2 x 1e-7, its residual tighter
    assert rel_err(X2, x0[perm]) <= 1e-3
    r_gpu = np.linalg.norm(ref2["b"] - A2 @ X2[inv], axis=0)
    r_o = np.linalg.norm(ref2["b"] - A2 @ x0, axis=0)
    assert np.all(np.abs(r_gpu - r_o) <= 1e-3 * r_o + 1e-6 * np.linalg.norm(ref2["b"], axis=0))
    assert np.all(r_o < 0.9 * np.linalg.norm(ref2["b"], axis=0))
    P.close()


@pytest.mark.parametrize("precision,rtol,tol", [(0, 1e-12, 1e-8), (1, 1e-9, 1e-6), (2, 1e-9, 1e-6)])
def test_recycled_solve_matches_direct_oracle(lib, chamber, precision, rtol, tol):
    mesh, eps, eps2, tx, rx, M, topo, perm, ref2 = chamber
    rng = np.random.default_rng(22)
    S_meas = ref2["S"] * (1 + 0.1 * rng.standard_normal(ref2["S"].shape))
    J_o, grad_o, extra = O.misfit_and_gradient(mesh.xyz, topo, eps2, FREQ, tx, rx, S_meas, fwd=ref2)
    its = {}
    for rec in (0, 1):
        P = lib.Problem(M, eps, FREQ, n_sub=6, precision=precision, recycle=rec, rtol=rtol, max_iter=300)
        P.forward_solve(tx, rx)
        P.misfit_and_gradient(S_meas)
        P.update_eps(eps2)
        S = P.forward_solve(tx, rx)
        its[rec] = P.info.iters_max
        assert P.info.n_converged == tx.shape[0]
        U = P.fields_host(0)
        assert col_rel_err(U, ref2["U"][perm]).max() <= tol
        assert rel_err(S, ref2["S"]) <= tol
        J, grad = P.misfit_and_gradient(S_meas)
        assert abs(J - J_o) <= tol * abs(J_o)
        assert rel_err(grad, grad_o) <= tol
        assert col_rel_err(P.fields_host(1), extra["Lam"][perm]).max() <= tol
        P.close()
    assert its[1] < its[0], its


def test_same_system_again_starts_from_its_solution(lib, chamber):
    mesh, eps, eps2, tx, rx, M, topo, perm, ref2 = chamber
    P = lib.Problem(M, eps2, FREQ, n_sub=6, precision=1, recycle=1, rtol=1e-6, max_iter=300)
    P.forward_solve(tx, rx)
    first = P.info.iters_max
    P.forward_solve(tx, rx)
    assert P.info.iters_max <= 1 < first
    assert col_rel_err(P.fields_host(0), ref2["U"][perm]).max() <= 1e-5
    P.close()


def test_recycling_edge_cases(lib, chamber):
    """A changed transmitter count does not recycle (different block shape) and
    still solves; recycling composes with the true block solver; one column."""
    mesh, eps, eps2, tx, rx, M, topo, perm, ref2 = chamber
    P = lib.Problem(M, eps, FREQ, n_sub=6, precision=0, recycle=1, block_krylov=1, rtol=1e-12, max_iter=300)
    P.forward_solve(tx[:3], rx)
    P.update_eps(eps2)
    S = P.forward_solve(tx, rx)  # 6 columns after 3: starts from zero
    assert P.info.n_converged == tx.shape[0] and P.info.iters_max > 0
    assert col_rel_err(P.fields_host(0), ref2["U"][perm]).max() <= 1e-8
    assert rel_err(S, ref2["S"]) <= 1e-8
    first = P.info.iters_max
    S = P.forward_solve(tx, rx)  # same 6 columns again: recycled into the block solver
    assert P.info.iters_max < first
    assert col_rel_err(P.fields_host(0), ref2["U"][perm]).max() <= 1e-8
    P.close()
    P = lib.Problem(M, eps2, FREQ, n_sub=6, precision=1, recycle=1, block_krylov=1, rtol=1e-9, max_iter=300)
    for _ in range(2):
        S = P.forward_solve(tx[2:3], rx)
        assert P.info.n_converged == 1
        assert col_rel_err(P.fields_host(0), ref2["U"][perm][:, 2:3]).max() <= 1e-6
    P.close()


@pytest.mark.parametrize("precision,rtol,tol", [(0, 1e-12, 1e-8), (1, 1e-9, 1e-6)])
def test_adjoint_recycles_forward_solutions(lib, chamber, precision, rtol, tol):
    """Receivers = transmitters: the adjoint right-hand sides lie in the span of
    the forward ones, so the adjoint solutions lie in the span of the forward
    solutions, and the first adjoint solve (no previous adjoint) starts next to
    them (to the accuracy of the FP32 projection)."""
    mesh, eps, eps2, tx, rx, M, topo, perm, ref2 = chamber
    rng = np.random.default_rng(23)
    S_meas = ref2["S"] * (1 + 0.1 * rng.standard_normal(ref2["S"].shape))
    J_o, grad_o, extra = O.misfit_and_gradient(mesh.xyz, topo, eps2, FREQ, tx, rx, S_meas, fwd=ref2)
    its = {}
    for rec in (0, 1):
        P = lib.Problem(M, eps2, FREQ, n_sub=6, precision=precision, recycle=rec, rtol=rtol, max_iter=300)
        P.forward_solve(tx, rx)
        J, grad = P.misfit_and_gradient(S_meas)
        its[rec] = P.info.iters_max
        assert abs(J - J_o) <= tol * abs(J_o)
        assert rel_err(grad, grad_o) <= tol
        assert col_rel_err(P.fields_host(1), extra["Lam"][perm]).max() <= tol
        P.close()
    # the FP32 projection leaves ~1e-7 of the residual: a few steps remain at these tolerances
    assert its[1] <= its[0] // 2, its


@pytest.mark.parametrize("precision,rtol,tol", [(0, 1e-12, 1e-8), (1, 1e-9, 1e-6)])
def test_factor_reuse_solves_the_new_system(lib, chamber, precision, rtol, tol):
    """factor_reuse = 1: the first eps_r update keeps the previous factors as
    the preconditioner of the new operator, the second refactors; both solves
    match the direct oracle solution of the new system."""
    mesh, eps, eps2, tx, rx, M, topo, perm, ref2 = chamber
    P = lib.Problem(M, eps, FREQ, n_sub=6, precision=precision, factor_reuse=1, rtol=rtol, max_iter=300)
    P.forward_solve(tx, rx)
    its = []
    for _ in range(2):
        P.update_eps(eps2)
        S = P.forward_solve(tx, rx)
        assert P.info.n_converged == tx.shape[0]
        its.append(P.info.iters_max)
        assert col_rel_err(P.fields_host(0), ref2["U"][perm]).max() <= tol
        assert rel_err(S, ref2["S"]) <= tol
    assert its[1] <= its[0], its  # the refactored preconditioner is the exact one
    P.close()
    with pytest.raises(lib.MwiError) as e:
        lib.Problem(M, eps, FREQ, n_sub=6, factor_reuse=-1)
    assert e.value.status == lib.MWI_EINVAL


def test_recycling_order2(lib):
    """Second-order elements: recycled solves of a perturbed system against the
    direct oracle (mixed path, rtol 1e-9 -> <= 1e-6)."""
    from tests._helpers import cube_case
    mesh, eps, tx, rx = cube_case(4)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag, order=2)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 2)
    kind, verts = M.dof_keys()
    perm = key_perm(kind, verts, topo)
    eps2 = eps * (1 + 0.03 * np.random.default_rng(24).uniform(-1, 1, mesh.nt))
    ref2 = O.forward(mesh.xyz, topo, eps2, FREQ, tx, rx)
    P = lib.Problem(M, eps, FREQ, n_sub=3, precision=1, recycle=1, rtol=1e-9, max_iter=300)
    P.forward_solve(tx, rx)
    P.update_eps(eps2)
    S = P.forward_solve(tx, rx)
    assert P.info.n_converged == tx.shape[0]
    assert col_rel_err(P.fields_host(0), ref2["U"][perm]).max() <= 1e-6
    assert rel_err(S, ref2["S"]) <= 1e-6
    P.close()
    M.close()


@pytest.mark.parametrize("precision,rtol,tol", [(0, 1e-12, 1e-8), (1, 1e-9, 1e-6)])
def test_recycling_across_nearby_frequencies(lib, chamber, precision, rtol, tol):
    """The solutions at 1 GHz, handed to the problem at 1.02 GHz
    (mwi_recycle_from), start its forward and adjoint solves: the results
    match the direct oracle at 1.02 GHz, in fewer iterations than from zero."""
    mesh, eps, eps2, tx, rx, M, topo, perm, ref2 = chamber
    f2 = 1.02e9
    P1 = lib.Problem(M, eps, FREQ, n_sub=6, precision=precision, rtol=rtol, max_iter=400)
    P1.forward_solve(tx, rx)
    S1 = P1.forward_solve(tx, rx)
    P1.misfit_and_gradient(S1 * 0.9)
    cold = lib.Problem(M, eps, f2, n_sub=6, precision=precision, rtol=rtol, max_iter=400)
    cold.forward_solve(tx, rx)
    it_cold = cold.info.iters_max
    S_c = cold.forward_solve(tx, rx)
    J_c, g_c = cold.misfit_and_gradient(S_c * 0.9)
    it_cold_adj = cold.info.iters_max
    warm = lib.Problem(M, eps, f2, n_sub=6, precision=precision, rtol=rtol, max_iter=400, recycle=1)
    warm.recycle_from(P1)
    S = warm.forward_solve(tx, rx)
    assert warm.info.iters_max < it_cold, (warm.info.iters_max, it_cold)
    ref = O.forward(mesh.xyz, topo, eps, f2, tx, rx)
    assert col_rel_err(warm.fields_host(0), ref["U"][perm]).max() <= tol
    assert rel_err(S, ref["S"]) <= tol
    J, g = warm.misfit_and_gradient(S * 0.9)
    J_o, g_o, _ = O.misfit_and_gradient(mesh.xyz, topo, eps, f2, tx, rx, S * 0.9, fwd=ref)
    assert abs(J - J_o) <= tol * abs(J_o) and rel_err(g, g_o) <= tol
    assert warm.info.iters_max <= it_cold_adj
    # refused without recycle = 1, or from a problem without solutions
    with pytest.raises(lib.MwiError):
        cold.recycle_from(P1)
    fresh = lib.Problem(M, eps, FREQ, n_sub=6, precision=precision, recycle=1)
    with pytest.raises(lib.MwiError):
        warm.recycle_from(fresh)
    for P in (P1, cold, warm, fresh):
        P.close()
