"""GPU parity of the nodal (P1) permittivity parameter (the piecewise-linear
parameter of Section 6.3: kappa varies inside every tet in the mass term) with
the gradient penalty and the normalised misfit (Eq. defJ2), through the C ABI,
against the oracle (oracle/p1.py).

Tolerances: the operator is the same sums in another order (closed-form
vertex masses against quadrature, <= 1e-13 relative); fields, S, the full
objective and its vertex gradient with the FP64 path solved to rtol 1e-12:
<= 1e-8 relative; the mixed path at rtol 1e-9: <= 1e-6.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from oracle import p1
from tests._helpers import FREQ, chamber_case, col_rel_err, cube_case, key_perm, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    return mwi


def _kappa(nv, seed, spread=5.0):
    rng = np.random.default_rng(seed)
    return 44 - 20j + rng.uniform(-spread, spread, nv) + 1j * rng.uniform(-spread / 2, spread / 2, nv)


@pytest.mark.parametrize("order", [1, 2])
def test_p1_operator_matches_oracle(lib, order):
    mesh, eps, tx, rx = cube_case(4 if order == 2 else 6)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag, order=order)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    perm = key_perm(*M.dof_keys(), topo)
    P = lib.Problem(M, eps, FREQ, n_sub=4)
    kap = _kappa(mesh.nv, 11)
    P.update_kappa(torch.from_numpy(kap).cuda())
    rp, col, val = P.matrix_csr()
    A_l = sp.csr_matrix((val, col, rp), shape=(M.ndof, M.ndof))
    Pm = sp.csr_matrix((np.ones(M.ndof), (np.arange(M.ndof), perm)), shape=(M.ndof, M.ndof))
    A_lo = (Pm.T @ A_l @ Pm).tocsr()
    A_o = p1.assemble_system_p1(mesh.xyz, topo, kap, FREQ)
    assert abs(A_lo - A_o).max() <= 1e-13 * abs(A_o).max()
    assert abs(A_l - A_l.T).max() == 0.0
    # a P0 update leaves nodal-parameter mode: the operator is the P0 one again
    P.update_eps(eps)
    rp, col, val = P.matrix_csr()
    A_l = sp.csr_matrix((val, col, rp), shape=(M.ndof, M.ndof))
    A_0 = O.assemble_system(mesh.xyz, topo, eps, FREQ)
    assert abs((Pm.T @ A_l @ Pm) - A_0).max() <= 1e-13 * abs(A_0).max()
    P.close()
    M.close()


def test_p1_objective_matches_oracle(lib):
    from paper_1607_02573_gb300.autograd import normalised_weights, p1_objective
    mesh, eps, tx, rx = cube_case(6)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    perm = key_perm(*M.dof_keys(), topo)
    eps_empty = np.full(mesh.nt, 44 - 20j)
    P = lib.Problem(M, eps_empty, FREQ, n_sub=4, precision=0, rtol=1e-12, max_iter=400)
    w = normalised_weights(P, eps_empty, tx, rx)
    w_o = p1.empty_chamber_weights(mesh.xyz, topo, eps_empty, FREQ, tx, rx)
    assert rel_err(w, w_o) <= 1e-8
    Mv = p1.vertex_mass_matrices(mesh.xyz, topo)
    S_meas = p1.forward_p1(mesh.xyz, topo, _kappa(mesh.nv, 12, 6.0), FREQ, tx, rx, Mv=Mv)["S"]
    kap = _kappa(mesh.nv, 13, 1.0)
    alpha = 1e-3
    phi, g = p1_objective(P, torch.from_numpy(kap).cuda(), tx, rx, S_meas, w, alpha)
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    phi_o, g_o, ex = p1.objective_p1(mesh.xyz, topo, kap, FREQ, tx, rx, S_meas, w_o, alpha, K, Mv=Mv)
    assert abs(phi - phi_o) <= 1e-8 * abs(phi_o)
    assert rel_err(g.cpu().numpy(), g_o) <= 1e-8
    U = P.fields_host(0)
    Uo = ex["U"][perm]
    assert col_rel_err(U, Uo).max() <= 1e-8
    Lam = P.fields_host(1)
    assert col_rel_err(Lam, ex["Lam"][perm]).max() <= 1e-8
    # the P0 gradient call refuses a problem in nodal-parameter mode
    with pytest.raises(lib.MwiError) as e:
        P.misfit_and_gradient(S_meas, w)
    assert e.value.status == lib.MWI_ESTATE
    P.close()
    M.close()


def test_p1_objective_mixed_path(lib):
    """The mixed path on the chamber against the oracle at rtol 1e-9, and its
    vertex gradient against central differences of its own objective."""
    from paper_1607_02573_gb300.autograd import p1_objective
    mesh, eps, tx, rx = chamber_case(12, 11, n_ant=8)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    P = lib.Problem(M, eps, FREQ, n_sub=8, precision=1, rtol=1e-9, max_iter=400)
    rng = np.random.default_rng(13)
    S_meas = P.forward_solve(tx, rx) * (1 + 0.05 * rng.standard_normal((tx.shape[0], rx.shape[0])))
    kap_h = np.full(mesh.nv, 44 - 20j) + rng.uniform(-2, 2, mesh.nv)
    kap = torch.from_numpy(kap_h).cuda()
    alpha = 1e-2
    phi, g = p1_objective(P, kap, tx, rx, S_meas, None, alpha)
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    Mv = p1.vertex_mass_matrices(mesh.xyz, topo)
    phi_o, g_o, _ = p1.objective_p1(mesh.xyz, topo, kap_h, FREQ, tx, rx, S_meas, None, alpha, K, Mv=Mv)
    assert abs(phi - phi_o) <= 1e-6 * abs(phi_o)
    g = g.cpu().numpy()
    assert rel_err(g, g_o) <= 1e-6
    P2 = lib.Problem(M, eps, FREQ, n_sub=8, precision=1, rtol=1e-11, max_iter=400)
    phi2, g2 = p1_objective(P2, kap, tx, rx, S_meas, None, alpha)
    g2 = g2.cpu().numpy()
    scale = np.abs(g2).max()
    cand = np.argsort(-np.abs(g2))[:200]
    for v in rng.choice(cand, 3, replace=False):
        for direction, comp in ((1.0, g2[v].real), (1j, g2[v].imag)):
            h = 1e-4 * abs(complex(kap[v]))
            kp = kap.clone(); kp[v] += direction * h
            km = kap.clone(); km[v] -= direction * h
            fd = (p1_objective(P2, kp, tx, rx, S_meas, None, alpha)[0] -
                  p1_objective(P2, km, tx, rx, S_meas, None, alpha)[0]) / (2 * h)
            assert abs(fd - comp) <= 1e-5 * scale + 1e-4 * abs(comp), (v, direction, fd, comp)
    P2.close()
    P.close()
    M.close()


def test_p1_rejects_bad_input(lib):
    mesh, eps, tx, rx = cube_case(4)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = lib.Problem(M, eps, FREQ, n_sub=2)
    kap = torch.from_numpy(_kappa(mesh.nv, 3)).cuda()
    kap[5] = complex(float("nan"), 0.0)
    with pytest.raises(lib.MwiError) as e:
        P.update_kappa(kap)
    assert e.value.status == lib.MWI_EINVAL
    with pytest.raises(lib.MwiError) as e:
        lib.normalised_weights(np.array([[1.0, 0.0]]))
    assert e.value.status == lib.MWI_EINVAL
    # gradient before any nodal parameter
    P.forward_solve(tx, rx)
    with pytest.raises(lib.MwiError) as e:
        P.misfit_and_gradient_kappa(np.zeros((4, 4)), None, 0.0)
    assert e.value.status == lib.MWI_ESTATE
    P.close()
    M.close()
