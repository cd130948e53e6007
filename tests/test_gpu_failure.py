"""Failure paths of the C ABI, made on the host (no GPU fault is provoked):

* a solve that hits max_iter returns MWI_ENOTCONV and still fills S, J, the
  gradient and the info struct (resid_max above rtol);
* a non-finite eps_r through the host and the device entry points returns
  MWI_EINVAL before anything changes (the problem keeps its operator);
* calls out of order return MWI_ESTATE (gradient before a forward solve, a
  mesh destroyed while a problem holds it);
* a lossless region (Im eps_r = 0 on some tets) voids the premise that makes
  every pivot of the unpivoted LDL^T non-zero; the solve must still reach the
  oracle's solution, the factorisation reporting any perturbed pivot.
"""

import ctypes as C

import numpy as np
import pytest

import oracle as O
from tests._helpers import FREQ, col_rel_err, cube_case, key_perm, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    return mwi


@pytest.mark.parametrize("precision", [0, 1])
def test_max_iter_gives_enotconv_with_filled_outputs(lib, precision):
    mesh, eps, tx, rx = cube_case(6)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = lib.Problem(M, eps, FREQ, n_sub=8, precision=precision, rtol=1e-12, max_iter=2)
    S_out = np.full((len(rx), len(tx)), np.nan + 0j)
    t, r = lib._antennas(tx), lib._antennas(rx)
    info = lib.mwi_solve_info()
    st = lib.mwi_forward_solve(P.h, t, len(t), r, len(r), lib._ptr(S_out.view(np.float64), C.c_double),
                               C.byref(info))
    assert st == lib.MWI_ENOTCONV
    assert b"rtol" in lib.mwi_last_error()
    assert np.all(np.isfinite(S_out)) and np.abs(S_out).max() > 0
    assert info.resid_max > 1e-12 and info.n_converged < len(tx) and info.iters_max <= 2
    S = S_out.T
    J, grad = P.misfit_and_gradient(S * 1.1, allow_notconv=True)
    assert P.info.resid_max > 1e-12
    assert np.isfinite(J) and J > 0 and np.all(np.isfinite(grad)) and np.abs(grad).max() > 0
    P.close()
    M.close()


def test_nonfinite_eps_is_rejected_on_host_and_device(lib):
    mesh, eps, tx, rx = cube_case(4)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    bad = eps.copy()
    bad[7] = complex(np.nan, -20.0)
    for make in (lambda e: lib.Problem(M, e, FREQ, n_sub=2),
                 lambda e: lib.Problem(M, torch.from_numpy(e).cuda(), FREQ, n_sub=2)):
        with pytest.raises(lib.MwiError) as err:
            make(bad)
        assert err.value.status == lib.MWI_EINVAL
    P = lib.Problem(M, eps, FREQ, n_sub=2, precision=0, rtol=1e-12)
    S0 = P.forward_solve(tx, rx)
    inf = eps.copy()
    inf[3] = complex(-20.0, np.inf)
    for upd in (lambda e: P.update_eps(e), lambda e: P.update_eps(torch.from_numpy(e).cuda())):
        with pytest.raises(lib.MwiError) as err:
            upd(inf)
        assert err.value.status == lib.MWI_EINVAL
        assert b"not finite" in lib.mwi_last_error()
    # the operator is unchanged
    S1 = P.forward_solve(tx, rx)
    assert rel_err(S1, S0) <= 1e-12
    P.close()
    M.close()


def test_calls_out_of_order_give_estate(lib):
    mesh, eps, tx, rx = cube_case(4)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = lib.Problem(M, eps, FREQ, n_sub=2)
    with pytest.raises(lib.MwiError) as err:
        P.misfit_and_gradient(np.zeros((4, 4)))
    assert err.value.status == lib.MWI_ESTATE
    assert lib.mwi_mesh_destroy(M.h) == lib.MWI_ESTATE
    P.close()
    M.close()


@pytest.mark.parametrize("precision,rtol,tol", [(0, 1e-12, 1e-8), (1, 1e-9, 1e-6)])
def test_lossless_region_solves_to_the_oracle(lib, precision, rtol, tol):
    mesh, eps, tx, rx = cube_case(8)
    c = mesh.xyz[mesh.tet].mean(axis=1)
    lossless = np.linalg.norm(c - 0.05, axis=1) < 0.03
    assert lossless.sum() > 100
    eps = eps.copy()
    eps[lossless] = 4.0 + 0.0j  # a dielectric phantom without loss
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    perm = key_perm(*M.dof_keys(), topo)
    P = lib.Problem(M, eps, FREQ, n_sub=8, precision=precision, rtol=rtol, max_iter=400)
    S = P.forward_solve(tx, rx)
    assert P.info.n_perturbed >= 0
    ref = O.forward(mesh.xyz, topo, eps, FREQ, tx, rx)
    assert col_rel_err(P.fields_host(0), ref["U"][perm]).max() <= tol
    assert rel_err(S, ref["S"]) <= tol
    P.close()
    M.close()
