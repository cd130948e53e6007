"""Full-size check on the bench workload (402,444-tet chamber, 32 antennas,
64 subdomains, mixed precision, rtol 1e-6 -- the configuration bench.py times).

The direct oracle cannot factor 458k complex DOFs in seconds, so the result
is checked through properties that hold at any size, evaluated with the
oracle's own assembly: the true residual ||b_j - A u_j|| / ||b_j|| of every
column (A and b assembled by the oracle, u mapped through the DOF keys), the
reciprocity S = S^T of the bilinear form, and, on sampled tets, the gradient
formula of Section 5 evaluated by the oracle on the returned state and
adjoint fields.
"""

import numpy as np
import pytest

import oracle as O
from tests._helpers import FREQ, key_perm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fullsize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas
    mesh = chamber_mesh(45, 42)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    ants = antenna_array(ring_antennas(32))
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = mwi.Problem(M, torch.from_numpy(eps).cuda(), FREQ, n_sub=64, precision=1, rtol=1e-6)
    S = P.forward_solve(ants, ants)
    info = P.info.as_dict()
    U = P.fields_host(0)
    rng = np.random.default_rng(3)
    S_meas = S * (1 + 0.05 * rng.standard_normal(S.shape))
    J, grad = P.misfit_and_gradient(S_meas)
    Lam = P.fields_host(1)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    kind, verts = M.dof_keys()
    perm = key_perm(kind, verts, topo)
    P.close()
    M.close()
    return dict(mesh=mesh, eps=eps, ants=ants, S=S, U=U, Lam=Lam, J=J, grad=grad, info=info, topo=topo,
                perm=perm, S_meas=S_meas)


def test_every_column_meets_rtol_with_oracle_operator(fullsize):
    d = fullsize
    assert d["info"]["n_converged"] == 32
    topo = d["topo"]
    A = O.assemble_system(d["mesh"].xyz, topo, d["eps"], FREQ)
    tdof, tsgn = O.antenna_edges(d["mesh"].xyz, topo, d["ants"])
    b = O.build_rhs(topo.ndof, tdof, tsgn, d["ants"][:, 6] + 1j * d["ants"][:, 7], FREQ)
    u = np.empty_like(d["U"])
    u[d["perm"]] = d["U"]
    r = np.linalg.norm(A @ u - b, axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 1.05e-6, r
    # S from the oracle's receiver map and the returned fields
    S_o = O.s_matrix(u, tdof, tsgn)
    assert np.abs(S_o - d["S"]).max() <= 1e-12 * np.abs(S_o).max()


def test_reciprocity_at_full_size(fullsize):
    S = fullsize["S"]
    assert np.linalg.norm(S - S.T) / np.linalg.norm(S) <= 1e-5


def test_adjoint_residual_and_sampled_gradient(fullsize):
    d = fullsize
    topo = d["topo"]
    mesh = d["mesh"]
    A = O.assemble_system(mesh.xyz, topo, d["eps"], FREQ)
    rdof, rsgn = O.antenna_edges(mesh.xyz, topo, d["ants"])
    J, r = O.misfit(d["S"], d["S_meas"])
    assert abs(J - d["J"]) <= 1e-10 * J
    g = O.adjoint_rhs(topo.ndof, r, None, rdof, rsgn)
    lam = np.empty_like(d["Lam"])
    lam[d["perm"]] = d["Lam"]
    res = np.linalg.norm(A @ lam - g, axis=0) / np.linalg.norm(g, axis=0)
    assert res.max() <= 1.05e-6, res
    u = np.empty_like(d["U"])
    u[d["perm"]] = d["U"]
    rng = np.random.default_rng(0)
    owners = np.unique(topo.face_tets[topo.face_tag == 2, 0])
    tets = np.concatenate([rng.choice(mesh.nt, 40, replace=False), owners[:10]])
    full = O.gradient(mesh.xyz, topo, d["eps"], FREQ, u, lam)
    assert np.abs(full[tets] - d["grad"][tets]).max() <= 1e-9 * np.abs(full).max()


@pytest.fixture(scope="module")
def inversion_setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    from synthetic import add_noise, antenna_array, chamber_mesh, chamber_target_eps, ring_antennas
    mesh = chamber_mesh(45, 42)
    target = chamber_target_eps(mesh.xyz, mesh.tet)
    ants = antenna_array(ring_antennas(32))
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = mwi.Problem(M, target, FREQ, n_sub=64, precision=1, rtol=1e-10)
    S_meas = add_noise(P.forward_solve(ants, ants), eta=0.01, seed=1234)
    yield dict(mesh=mesh, ants=ants, M=M, P=P, S_meas=S_meas)
    P.close()
    M.close()


def test_fullsize_gradient_matches_finite_differences(inversion_setup):
    """Adjoint gradient of J on the full chamber against central differences of
    the GPU's own J on 10 seeded random tets (real part) and 3 (imaginary part)."""
    d = inversion_setup
    mesh, ants, P, S_meas = d["mesh"], d["ants"], d["P"], d["S_meas"]
    eps0 = np.full(mesh.nt, 44 - 20j)
    P.update_eps(eps0)
    P.forward_solve(ants, ants)
    J0, grad = P.misfit_and_gradient(S_meas)
    rng = np.random.default_rng(5)
    tets = rng.choice(mesh.nt, 10, replace=False)
    scale = np.abs(grad).max()

    def J_at(e):
        P.update_eps(e)
        P.forward_solve(ants, ants)
        return P.misfit(S_meas)

    for q, t in enumerate(tets):
        for direction, comp in ((1.0, grad[t].real), (1j, grad[t].imag)):
            if direction == 1j and q >= 3:
                continue
            h = 1e-4 * abs(eps0[t])
            ep = eps0.copy(); ep[t] += direction * h
            em = eps0.copy(); em[t] -= direction * h
            fd = (J_at(ep) - J_at(em)) / (2 * h)
            assert abs(fd - comp) <= 1e-5 * scale + 1e-4 * abs(comp), (t, direction, fd, comp)


def test_fullsize_lbfgs_reduces_misfit(inversion_setup):
    """Ten L-BFGS iterations from the homogeneous gel towards the two-inclusion
    target (1 % noise): the misfit must drop substantially."""
    from paper_1607_02573_gb300.autograd import lbfgs_invert
    d = inversion_setup
    mesh, ants, P, S_meas = d["mesh"], d["ants"], d["P"], d["S_meas"]
    eps0 = np.full(mesh.nt, 44 - 20j)
    rec, values = lbfgs_invert(P, eps0, ants, ants, S_meas, iters=10)
    assert np.all(np.isfinite(values))
    assert values[-1] < 0.2 * values[0], values
