"""GPU parity of the nodal (P1) permittivity parameter with the gradient
penalty and the normalised misfit (Eq. defJ2; P1 parameter of Section 6.3),
through the C ABI, against the oracle (oracle/p1.py).

Tolerances: the centroid sampling and the spreading are the same sums in a
different order (<= 1e-14 relative); the full objective with the FP64 path
solved to rtol 1e-12: <= 1e-8 relative, as for the per-tet gradient.
"""

import numpy as np
import pytest

import oracle as O
from oracle import p1
from tests._helpers import FREQ, chamber_case, cube_case, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    return mwi


def test_sampling_spreading_and_penalty_match_oracle(lib):
    mesh, eps, tx, rx = cube_case(6)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    rng = np.random.default_rng(11)
    kap = 44 - 20j + rng.uniform(-5, 5, mesh.nv) + 1j * rng.uniform(-2, 2, mesh.nv)
    g_t = rng.standard_normal(mesh.nt) + 1j * rng.standard_normal(mesh.nt)
    kd = torch.from_numpy(kap).cuda()
    eps_d = M.p1_tet_eps(kd)
    assert rel_err(eps_d.cpu().numpy(), p1.p1_to_tet(mesh.tet, kap)) <= 1e-14
    alpha = 0.37
    g_v, R = M.p1_gradient(torch.from_numpy(g_t).cuda(), kd, alpha)
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    R_o, gR_o = p1.regularisation(K, kap, alpha)
    ref = p1.p1_spread(mesh.tet, mesh.nv, g_t) + gR_o
    assert rel_err(g_v.cpu().numpy(), ref) <= 1e-13
    assert abs(R - R_o) <= 1e-12 * abs(R_o)
    # constants carry no penalty
    _, R0 = M.p1_gradient(torch.from_numpy(g_t).cuda(), torch.full((mesh.nv,), 5.0 - 1.0j,
                                                                   dtype=torch.complex128, device="cuda"), alpha)
    assert abs(R0) <= 1e-12 * abs(R_o)
    M.close()


def test_p1_objective_matches_oracle(lib):
    from paper_1607_02573_gb300.autograd import normalised_weights, p1_objective
    mesh, eps, tx, rx = cube_case(6)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    rng = np.random.default_rng(12)
    kap_true = 44 - 20j + rng.uniform(-6, 6, mesh.nv) + 1j * rng.uniform(-3, 3, mesh.nv)
    eps_empty = np.full(mesh.nt, 44 - 20j)
    P = lib.Problem(M, eps_empty, FREQ, n_sub=4, precision=0, rtol=1e-12, max_iter=400)
    w = normalised_weights(P, eps_empty, tx, rx)
    w_o = p1.empty_chamber_weights(mesh.xyz, topo, eps_empty, FREQ, tx, rx)
    assert rel_err(w, w_o) <= 1e-8
    S_meas = O.forward(mesh.xyz, topo, p1.p1_to_tet(mesh.tet, kap_true), FREQ, tx, rx)["S"]
    kap = np.full(mesh.nv, 44 - 20j) + rng.uniform(-1, 1, mesh.nv)
    alpha = 1e-3
    phi, g = p1_objective(P, torch.from_numpy(kap).cuda(), tx, rx, S_meas, w, alpha)
    K = p1.p1_stiffness(mesh.xyz, mesh.tet)
    phi_o, g_o = p1.objective_p1(mesh.xyz, topo, mesh.tet, kap, FREQ, tx, rx, S_meas, w_o, alpha, K)
    assert abs(phi - phi_o) <= 1e-8 * abs(phi_o)
    assert rel_err(g.cpu().numpy(), g_o) <= 1e-8
    P.close()
    M.close()


def test_p1_objective_finite_differences_mixed(lib):
    """The mixed path's P1 objective gradient against central differences of
    its own objective on the chamber, in Re and Im of kappa at sampled vertices."""
    from paper_1607_02573_gb300.autograd import p1_objective
    mesh, eps, tx, rx = chamber_case(12, 11, n_ant=8)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = lib.Problem(M, eps, FREQ, n_sub=8, precision=1, rtol=1e-11, max_iter=400)
    rng = np.random.default_rng(13)
    S_meas = P.forward_solve(tx, rx) * (1 + 0.05 * rng.standard_normal((tx.shape[0], rx.shape[0])))
    kap = torch.full((mesh.nv,), 44 - 20j, dtype=torch.complex128, device="cuda")
    alpha = 1e-2
    phi, g = p1_objective(P, kap, tx, rx, S_meas, None, alpha)
    g = g.cpu().numpy()
    scale = np.abs(g).max()
    # vertices inside the chamber with a non-negligible gradient
    cand = np.argsort(-np.abs(g))[:200]
    for v in rng.choice(cand, 3, replace=False):
        for direction, comp in ((1.0, g[v].real), (1j, g[v].imag)):
            h = 1e-4 * abs(complex(kap[v]))
            kp = kap.clone(); kp[v] += direction * h
            km = kap.clone(); km[v] -= direction * h
            fd = (p1_objective(P, kp, tx, rx, S_meas, None, alpha)[0] -
                  p1_objective(P, km, tx, rx, S_meas, None, alpha)[0]) / (2 * h)
            assert abs(fd - comp) <= 1e-5 * scale + 1e-4 * abs(comp), (v, direction, fd, comp)
    P.close()
    M.close()
