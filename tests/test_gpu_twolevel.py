"""GPU parity of the two-level ORAS (coarse space of Section 7) through the C ABI.

* the prolongation P and the Galerkin operator A_c = P^T A P against the
  oracle's CoarseSpace on a jittered, permuted fine chamber and an unjittered
  coarse one (P: the same midpoint rule, <= 1e-12 of max |P|; A_c: the same
  sums in another order, <= 1e-12 of max |A_c|), and again after an eps_r
  update (A_c follows the refactorisation);
* one application of the deflated two-level preconditioner against the
  oracle's: FP64 <= 1e-9 relative (two FP64 LDL^T factorisations, the dense
  coarse one against SuperLU); MIXED with FP32 factors, coarse solve on the
  3xTF32 mma engine, subdomain sweeps on the engine under test;
* with the fine mesh as its own coarse mesh, P = I, Q = A^{-1} and FGMRES stops
  after one iteration (a property of the method, not of the oracle);
* forward fields and S of a two-level solve against the direct oracle
  (FP64 rtol 1e-12 -> 1e-8; MIXED rtol 1e-9 -> 1e-6);
* removing the coarse space gives back the one-level results bit for bit;
  the allocation-free entry point refuses a problem with a coarse space; a
  second-order coarse mesh is refused.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import dd
from synthetic import chamber_mesh
from tests._helpers import FREQ, chamber_case, col_rel_err, cube_case, key_perm, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    return mwi


def _perm_matrix(perm):
    n = perm.size
    return sp.csr_matrix((np.ones(n), (np.arange(n), perm)), shape=(n, n))


def _case(lib, nsub=6, fine=(10, 9), coarse=(6, 5)):
    mesh, eps, tx, rx = chamber_case(*fine, n_ant=4, radius=0.08)
    cm = chamber_mesh(*coarse, jitter=0.0, permute=False)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    Mc = lib.Mesh(cm.xyz, cm.tet, cm.bface_tag)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    ct = O.build_topology(cm.tet, cm.bface_tag, cm.nv, 1)
    perm = key_perm(*M.dof_keys(), topo)
    cperm = key_perm(*Mc.dof_keys(), ct)
    part = dd.rcb_partition(mesh.xyz, mesh.tet, nsub)
    return dict(mesh=mesh, eps=eps, tx=tx, rx=rx, cm=cm, M=M, Mc=Mc, topo=topo, ct=ct, perm=perm, cperm=cperm,
                part=part, nsub=nsub)


def _oracle_cs(c, eps):
    mesh, topo = c["mesh"], c["topo"]
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ).tocsr()
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, c["part"], 1)
    oras = dd.ORAS(dec, dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ))
    return dd.CoarseSpace(mesh.xyz, topo, c["cm"].xyz, c["ct"], A, oras)


def _close(c, *problems):
    for P in problems:
        P.close()
    c["Mc"].close()
    c["M"].close()


def test_prolongation_and_coarse_operator_match_oracle(lib):
    c = _case(lib)
    P = lib.Problem(c["M"], c["eps"], FREQ, n_sub=c["nsub"], part=c["part"])
    P.set_coarse_space(c["Mc"])
    info = P.coarse_info()
    assert info["n_coarse"] == c["ct"].ndof and info["n_perturbed"] == 0
    cs = _oracle_cs(c, c["eps"])
    Pf, Pc = _perm_matrix(c["perm"]), _perm_matrix(c["cperm"])
    Pl, Acl = P.coarse_operator()
    # library order -> oracle order on both meshes
    P_lo = (Pf.T @ Pl @ Pc).tocsr()
    assert abs(P_lo - cs.P).max() <= 1e-12 * abs(cs.P).max()
    Ac_lo = (Pc.T @ Acl @ Pc).tocsr()
    assert abs(Ac_lo - cs.Ac).max() <= 1e-12 * abs(cs.Ac).max()
    # A_c follows an eps_r update
    eps2 = c["eps"] * (1.0 + 0.05 * np.random.default_rng(4).standard_normal(c["eps"].shape))
    P.update_eps(eps2)
    cs2 = _oracle_cs(c, eps2)
    Ac2 = (Pc.T @ P.coarse_operator()[1] @ Pc).tocsr()
    assert abs(Ac2 - cs2.Ac).max() <= 1e-12 * abs(cs2.Ac).max()
    assert abs(Ac2 - cs.Ac).max() > 1e-6 * abs(cs.Ac).max()
    _close(c, P)


@pytest.mark.parametrize("precision,engine,tol", [(0, 0, 1e-9), (1, 1, 1e-4), (1, 4, 1e-2)])
def test_two_level_apply_parity(lib, precision, engine, tol):
    c = _case(lib)
    P = lib.Problem(c["M"], c["eps"], FREQ, n_sub=c["nsub"], part=c["part"], precision=precision,
                    sweep_engine=engine)
    P.set_coarse_space(c["Mc"])
    cs = _oracle_cs(c, c["eps"])
    rng = np.random.default_rng(2)
    n = c["M"].ndof
    for m in (3, 8):
        X = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
        Y = P.oras_apply(torch.from_numpy(X).cuda()).cpu().numpy()
        inv = np.argsort(c["perm"])
        Xo = X[inv]
        Yo = np.stack([cs.apply(Xo[:, k]) for k in range(m)], axis=1)[c["perm"]]
        assert rel_err(Y, Yo) <= tol, (m, rel_err(Y, Yo))
    _close(c, P)


def test_fine_mesh_as_coarse_space_is_exact(lib):
    mesh, eps, tx, rx = cube_case(4)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    Mc = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = lib.Problem(M, eps, FREQ, n_sub=4, precision=0, rtol=1e-10)
    P.set_coarse_space(Mc)
    Pl, _ = P.coarse_operator()
    assert abs(Pl - sp.identity(M.ndof)).max() <= 1e-12
    P.forward_solve(tx, rx)
    assert P.info.iters_max == 1
    P.close()
    Mc.close()
    M.close()


@pytest.mark.parametrize("precision,engine,rtol,tol", [(0, 0, 1e-12, 1e-8), (1, 4, 1e-9, 1e-6), (2, 4, 1e-9, 1e-6)])
def test_two_level_forward_parity(lib, precision, engine, rtol, tol):
    c = _case(lib, nsub=8)
    P = lib.Problem(c["M"], c["eps"], FREQ, n_sub=c["nsub"], part=c["part"], precision=precision,
                    sweep_engine=engine, rtol=rtol)
    P.set_coarse_space(c["Mc"])
    S = P.forward_solve(c["tx"], c["rx"])
    U = P.fields_host(0)
    ref = O.forward(c["mesh"].xyz, c["topo"], c["eps"], FREQ, c["tx"], c["rx"])
    assert col_rel_err(U, ref["U"][c["perm"]]).max() <= tol
    assert rel_err(S, ref["S"]) <= tol
    _close(c, P)


def test_removing_the_coarse_space_restores_one_level(lib):
    c = _case(lib)
    kw = dict(n_sub=c["nsub"], part=c["part"], precision=1, sweep_engine=4, rtol=1e-9)
    P1 = lib.Problem(c["M"], c["eps"], FREQ, **kw)
    S1 = P1.forward_solve(c["tx"], c["rx"])
    it1 = P1.info.iters_max
    P2 = lib.Problem(c["M"], c["eps"], FREQ, **kw)
    P2.set_coarse_space(c["Mc"])
    S2 = P2.forward_solve(c["tx"], c["rx"])
    assert P2.info.iters_max <= it1
    assert rel_err(S2, S1) <= 1e-6
    X = torch.from_numpy(np.ones((c["M"].ndof, 2), dtype=np.complex128)).cuda()
    Y = torch.empty_like(X)
    with pytest.raises(lib.MwiError):
        lib.check(lib.mwi_oras_apply_device_noalloc(P2.h, X.data_ptr(), Y.data_ptr(), 2))
    P2.set_coarse_space(None)
    S3 = P2.forward_solve(c["tx"], c["rx"])
    assert np.array_equal(S3, S1) and P2.info.iters_max == it1
    _close(c, P1, P2)


def test_second_order_coarse_mesh_is_refused(lib):
    c = _case(lib)
    P = lib.Problem(c["M"], c["eps"], FREQ, n_sub=c["nsub"], part=c["part"])
    cm = c["cm"]
    Mc2 = lib.Mesh(cm.xyz, cm.tet, cm.bface_tag, order=2)
    with pytest.raises(lib.MwiError):
        P.set_coarse_space(Mc2)
    assert P.coarse_info()["n_coarse"] == 0
    Mc2.close()
    _close(c, P)
