"""torch.autograd.Function and L-BFGS driver (Section 5: the gradient by the
adjoint method feeds a quasi-Newton reconstruction).

* MisfitGrad: forward gives the oracle's J, backward gives the oracle's
  dJ/dRe + i dJ/dIm (PyTorch's convention for a real loss of a complex input);
* finite differences of the GPU's own J along random directions agree with the
  directional derivative from the backward pass;
* a few L-BFGS iterations reduce the misfit towards a target map.
"""

import numpy as np
import pytest

import oracle as O
from tests._helpers import FREQ, chamber_case, cube_case, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import autograd, mwi
    return mwi, autograd


def test_misfitgrad_matches_oracle(lib):
    mwi, ag = lib
    mesh, eps, tx, rx = cube_case(6)
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = mwi.Problem(M, eps, FREQ, n_sub=3, rtol=1e-12)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    ref = O.forward(mesh.xyz, topo, eps, FREQ, tx, rx)
    S_meas = ref["S"] * 1.1
    e = torch.tensor(eps, dtype=torch.complex128, requires_grad=True)
    J = ag.MisfitGrad.apply(e, P, tx, rx, S_meas, None)
    J.backward()
    J_o, g_o, _ = O.misfit_and_gradient(mesh.xyz, topo, eps, FREQ, tx, rx, S_meas, fwd=ref)
    assert abs(float(J.detach()) - J_o) <= 1e-8 * J_o
    assert rel_err(e.grad.numpy(), g_o) <= 1e-8
    P.close()


def test_directional_derivative_matches_finite_difference(lib):
    mwi, ag = lib
    mesh, eps, tx, rx = chamber_case(12, 11, n_ant=6)
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = mwi.Problem(M, eps, FREQ, n_sub=4, rtol=1e-12)
    S0 = P.forward_solve(tx, rx)
    S_meas = S0 * 0.95
    e = torch.tensor(eps, dtype=torch.complex128, requires_grad=True)
    J = ag.MisfitGrad.apply(e, P, tx, rx, S_meas, None)
    J.backward()
    g = e.grad.numpy()
    rng = np.random.default_rng(4)
    for _ in range(3):
        d = rng.standard_normal(mesh.nt) + 1j * rng.standard_normal(mesh.nt)
        h = 1e-4
        Jp = float(ag.MisfitGrad.apply(torch.tensor(eps + h * d), P, tx, rx, S_meas, None))
        Jm = float(ag.MisfitGrad.apply(torch.tensor(eps - h * d), P, tx, rx, S_meas, None))
        fd = (Jp - Jm) / (2 * h)
        an = float(np.sum(g.real * d.real + g.imag * d.imag))
        assert abs(fd - an) <= 1e-5 * abs(an) + 1e-12, (fd, an)
    P.close()


def test_lbfgs_reduces_misfit(lib):
    """Four L-BFGS iterations, with and without recycling of the previous
    evaluation's solutions: both reduce the misfit, and since every solve runs
    to rtol 1e-10 the two take the same path (same J values to 1e-6)."""
    mwi, ag = lib
    from synthetic import chamber_target_eps
    mesh, eps, tx, rx = chamber_case(12, 11, n_ant=8)
    target = chamber_target_eps(mesh.xyz, mesh.tet)
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    runs = {}
    for recycle in (0, 1):
        P = mwi.Problem(M, target, FREQ, n_sub=4, rtol=1e-10, precision=1, recycle=recycle)
        S_meas = P.forward_solve(tx, rx)
        eps0 = np.full(mesh.nt, 44 - 20j)
        rec, values = ag.lbfgs_invert(P, eps0, tx, rx, S_meas, iters=4)
        assert values[-1] < 0.5 * values[0]
        assert np.all(np.isfinite(rec))
        runs[recycle] = values
        P.close()
    assert len(runs[0]) == len(runs[1])
    assert np.allclose(runs[0], runs[1], rtol=1e-6, atol=0)
