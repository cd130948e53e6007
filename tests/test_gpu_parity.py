"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (complex128 results):
* assembly and SpMM: the same sums in a different order, <= 1e-13 relative;
* one ORAS application in FP64: <= 1e-10 relative (local LDL^T vs SuperLU
  on B_i with condition numbers up to ~1e4);
* FP64 path solved to rtol 1e-12: fields, S and gradient <= 1e-8 relative;
* MIXED path (FP32 subdomain factors) solved to rtol 1e-9: <= 1e-6 relative.
"""

import numpy as np
import pytest

import oracle as O
from oracle import dd
from tests._helpers import FREQ, chamber_case, col_rel_err, cube_case, key_perm, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    return mwi


_REF_CACHE = {}


def _oracle_reference(key, mesh, topo, eps, tx, rx, S_meas_scale=None):
    """Oracle forward solve and misfit/gradient for one case, computed once per module."""
    if key not in _REF_CACHE:
        ref = O.forward(mesh.xyz, topo, eps, FREQ, tx, rx)
        rng = np.random.default_rng(5)
        S_meas = ref["S"] * (1 + 0.2 * rng.standard_normal(ref["S"].shape))
        J_o, grad_o, extra = O.misfit_and_gradient(mesh.xyz, topo, eps, FREQ, tx, rx, S_meas, fwd=ref)
        _REF_CACHE[key] = (ref, S_meas, J_o, grad_o, extra)
    return _REF_CACHE[key]


def _setup(lib, case, order=1, **opts):
    mesh, eps, tx, rx = case
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag, order=order)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, order)
    kind, verts = M.dof_keys()
    perm = key_perm(kind, verts, topo)
    return mesh, eps, tx, rx, M, topo, perm


@pytest.mark.parametrize("order", [1, 2])
def test_matrix_and_spmm_parity(lib, order):
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, cube_case(4 if order == 2 else 8), order)
    P = lib.Problem(M, eps, FREQ, n_sub=4)
    A_o = O.assemble_system(mesh.xyz, topo, eps, FREQ).tocsr()
    rp, col, val = P.matrix_csr()
    import scipy.sparse as sp
    A_l = sp.csr_matrix((val, col, rp), shape=(M.ndof, M.ndof))
    # map library indices to oracle indices
    Pm = sp.csr_matrix((np.ones(M.ndof), (np.arange(M.ndof), perm)), shape=(M.ndof, M.ndof))
    A_lo = (Pm.T @ A_l @ Pm).tocsr()
    d = abs(A_lo - A_o).max()
    assert d <= 1e-13 * abs(A_o).max()
    assert abs(A_l - A_l.T).max() == 0.0
    rng = np.random.default_rng(0)
    m = 5
    X = rng.standard_normal((M.ndof, m)) + 1j * rng.standard_normal((M.ndof, m))
    Xd = torch.from_numpy(X).cuda()
    Y = P.spmm(Xd).cpu().numpy()
    Yo = np.empty_like(Y)
    Yo[:] = (A_o @ X[np.argsort(perm)])[perm]
    assert rel_err(Y, Yo) <= 1e-13
    P.close()


def test_partition_matches_oracle_rcb(lib):
    case = chamber_case(12, 11)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    P = lib.Problem(M, eps, FREQ, n_sub=8)
    part, nloc = P.decomposition(8)
    assert np.array_equal(part, dd.rcb_partition(mesh.xyz, mesh.tet, 8))
    P.close()


@pytest.mark.parametrize("m", [3, 6, 40])
@pytest.mark.parametrize("precision,engine,tol", [(0, 0, 1e-10), (1, 1, 2e-5), (1, 3, 2e-5), (1, 2, 5e-3),
                                                  (1, 4, 1e-2)])
def test_oras_apply_parity(lib, precision, engine, tol, m):
    """engine: complex FP32 sweeps on tensor cores with split TF32 operands (1),
    plain TF32 (2, about 1e-3 relative), CUDA cores (3), or tcgen05 TF32 with
    bulk-copied tiled panels (4: the tensor core truncates the FP32 operands
    to TF32, up to 2^-10 relative per operand; an odd column count gets one
    zero padding column).  m: columns -- odd, even, and two 32-column chunks
    with a ragged second one."""
    case = chamber_case(12, 11)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    part = dd.rcb_partition(mesh.xyz, mesh.tet, 6)
    P = lib.Problem(M, eps, FREQ, n_sub=6, part=part, precision=precision, sweep_engine=engine)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    oras = dd.ORAS(dec, dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ))
    rng = np.random.default_rng(1)
    X = rng.standard_normal((M.ndof, m)) + 1j * rng.standard_normal((M.ndof, m))
    Y = P.oras_apply(torch.from_numpy(X).cuda()).cpu().numpy()
    inv = np.argsort(perm)
    Yo = oras.apply(X[inv])[perm]
    assert rel_err(Y, Yo) <= tol
    P.close()


@pytest.mark.parametrize("case_name", ["cube", "chamber"])
@pytest.mark.parametrize("precision,engine,rtol,tol", [(0, 0, 1e-12, 1e-8), (1, 1, 1e-9, 1e-6), (1, 2, 1e-9, 1e-6),
                                                       (1, 3, 1e-9, 1e-6), (1, 4, 1e-9, 1e-6), (2, 1, 1e-9, 1e-6),
                                                       (2, 4, 1e-9, 1e-6)])
def test_forward_and_gradient_parity(lib, case_name, precision, engine, rtol, tol):
    case = cube_case(8) if case_name == "cube" else chamber_case(16, 15)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    n_sub = 4 if case_name == "cube" else 8
    P = lib.Problem(M, eps, FREQ, n_sub=n_sub, precision=precision, rtol=rtol, max_iter=400, sweep_engine=engine)
    S = P.forward_solve(tx, rx)
    info = P.info.as_dict()
    assert info["n_converged"] == tx.shape[0]
    ref, S_meas, J_o, grad_o, extra = _oracle_reference(case_name, mesh, topo, eps, tx, rx)
    U = P.fields_host(0)
    errs = col_rel_err(U, ref["U"][perm])
    assert errs.max() <= tol, errs
    assert rel_err(S, ref["S"]) <= tol
    # misfit and gradient against seeded synthetic measurements
    J, grad = P.misfit_and_gradient(S_meas)
    assert abs(J - J_o) <= tol * abs(J_o)
    assert rel_err(grad, grad_o) <= tol
    Lam = P.fields_host(1)
    assert col_rel_err(Lam, extra["Lam"][perm]).max() <= tol
    P.close()


@pytest.mark.parametrize("precision,restart,rtol,tol", [(0, 3, 1e-12, 1e-8), (1, 3, 1e-9, 1e-6), (2, 1, 1e-9, 1e-6)])
def test_restarted_solver_parity(lib, precision, restart, rtol, tol):
    """A short restart length forces several FGMRES cycles (each ends on the
    true residual and restarts from it; the nested variant's outer iteration
    needs few steps, so it restarts after every one): the converged fields must
    still match the oracle's direct solution."""
    case = chamber_case(16, 15)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    P = lib.Problem(M, eps, FREQ, n_sub=8, precision=precision, rtol=rtol, max_iter=400, restart=restart)
    S = P.forward_solve(tx, rx)
    info = P.info.as_dict()
    assert info["n_converged"] == tx.shape[0]
    assert info["iters_max"] > restart
    assert info["resid_max"] <= rtol
    ref, S_meas, J_o, grad_o, extra = _oracle_reference("chamber", mesh, topo, eps, tx, rx)
    U = P.fields_host(0)
    assert col_rel_err(U, ref["U"][perm]).max() <= tol
    assert rel_err(S, ref["S"]) <= tol
    P.close()


def test_reciprocity_and_weights(lib):
    case = chamber_case(14, 13, n_ant=6)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    P = lib.Problem(M, eps, FREQ, n_sub=8, rtol=1e-11)
    S = P.forward_solve(tx, rx)
    assert rel_err(S, S.T) <= 1e-9
    w = np.random.default_rng(2).uniform(0.5, 2.0, S.shape)
    S_meas = S * 0.9
    J, grad = P.misfit_and_gradient(S_meas, w=w)
    assert abs(J - 0.5 * np.sum(w * np.abs(S - S_meas) ** 2)) <= 1e-9 * J
    P.close()


@pytest.mark.parametrize("opts", [{}, {"block_krylov": 1}, {"recycle": 1}, {"precision": 1, "recycle": 1}])
def test_zero_misfit_gives_zero_gradient(lib, opts):
    """A zero adjoint right-hand side (zero misfit) gives Lambda = 0 and a zero
    gradient in every solver, twice in a row (the second adjoint solve recycles
    a zero block when recycle = 1)."""
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, cube_case(6))
    P = lib.Problem(M, eps, FREQ, n_sub=2, rtol=1e-10, **opts)
    for _ in range(2):
        S = P.forward_solve(tx, rx)
        J, grad = P.misfit_and_gradient(S)
        assert J == 0.0 and np.abs(grad).max() == 0.0
    P.close()


def test_errors_are_reported(lib):
    mesh, eps, tx, rx = cube_case(4)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = lib.Problem(M, eps, FREQ, n_sub=2)
    with pytest.raises(lib.MwiError) as e:
        P.misfit_and_gradient(np.zeros((4, 4), dtype=complex))
    assert e.value.status == lib.MWI_ESTATE
    # empty and oversized antenna sets are refused before any device work
    for t, r in [(tx[:0], rx), (tx, rx[:0]), (np.repeat(tx[:1], 4097, axis=0), rx)]:
        with pytest.raises(lib.MwiError) as e:
            P.forward_solve(t, r)
        assert e.value.status == lib.MWI_EINVAL
    with pytest.raises(lib.MwiError) as e:
        M.close()
    assert e.value.status == lib.MWI_ESTATE
    P.close()
    M.close()


@pytest.mark.parametrize("precision,rtol,tol", [(0, 1e-12, 1e-8), (1, 1e-9, 1e-6)])
def test_order2_forward_and_gradient_parity(lib, precision, rtol, tol):
    case = cube_case(4)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case, order=2)
    P = lib.Problem(M, eps, FREQ, n_sub=3, precision=precision, rtol=rtol, max_iter=300)
    S = P.forward_solve(tx, rx)
    ref = O.forward(mesh.xyz, topo, eps, FREQ, tx, rx)
    U = P.fields_host(0)
    assert col_rel_err(U, ref["U"][perm]).max() <= tol
    assert rel_err(S, ref["S"]) <= tol
    S_meas = ref["S"] * 0.8
    J, grad = P.misfit_and_gradient(S_meas)
    J_o, grad_o, _ = O.misfit_and_gradient(mesh.xyz, topo, eps, FREQ, tx, rx, S_meas, fwd=ref)
    assert abs(J - J_o) <= tol * abs(J_o)
    assert rel_err(grad, grad_o) <= tol
    P.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_columns_independent_of_block_width(lib, precision):
    """Every right-hand side keeps its own Krylov state, so a column's result is the
    same (bit for bit) whether it is solved alone, in a block of 3 or in one block."""
    case = chamber_case(12, 11, n_ant=8)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    res = []
    for mb in (64, 3, 1):
        P = lib.Problem(M, eps, FREQ, n_sub=4, precision=precision, rtol=1e-9, max_block=mb)
        S = P.forward_solve(tx, rx)
        J, grad = P.misfit_and_gradient(S * 0.9)
        res.append((S, J, grad))
        P.close()
    for S, J, grad in res[1:]:
        assert np.array_equal(S, res[0][0])
        assert np.array_equal(grad, res[0][2])


def _db_bins(S, S_o):
    a = np.abs(S_o)
    db = 20.0 * np.log10(a / a.max())
    rel = np.abs(S - S_o) / a
    return db, rel


@pytest.mark.parametrize("precision,engine,rtol", [(0, 0, 1e-12), (1, 4, 1e-9), (1, 2, 1e-9)])
def test_s_and_gradient_entrywise_by_db_bins(lib, precision, engine, rtol):
    """S entry by entry, binned by |S| in dB below its largest entry (the weak
    transmissions carry the image, paper Section 6.2), and the gradient tet by
    tet.  The solver bounds the error of every column relative to the column,
    so an entry X dB below the largest one can lose up to X/20 digits: the
    bound per bin is C rtol 10^(-lo/20), lo the bin's lower edge (the weakest
    entry for the last bin), C = 1e3 as in the normwise tolerances above; the
    gradient per tet is bounded by C rtol max|grad|."""
    case = chamber_case(16, 15)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    P = lib.Problem(M, eps, FREQ, n_sub=8, precision=precision, rtol=rtol, max_iter=400, sweep_engine=engine)
    S = P.forward_solve(tx, rx)
    ref, S_meas, J_o, grad_o, extra = _oracle_reference("chamber", mesh, topo, eps, tx, rx)
    S_o = ref["S"]
    db, rel = _db_bins(S, S_o)
    assert db.min() < -60.0, db.min()  # the case spans the three bins
    C = 1e3
    report = {}
    for hi, lo in ((0.0, -20.0), (-20.0, -60.0), (-60.0, float(db.min()))):
        sel = (db <= hi) & (db >= lo)
        assert sel.any()
        report[f"{hi:g}..{lo:.0f} dB"] = float(rel[sel].max())
        assert rel[sel].max() <= C * rtol * 10.0 ** (-lo / 20.0), report
    J, grad = P.misfit_and_gradient(S_meas)
    assert np.abs(grad - grad_o).max() <= C * rtol * np.abs(grad_o).max()
    P.close()


def test_antenna_map_reuse_follows_the_antennas(lib):
    """A forward solve with the same antennas as the previous one reuses the
    antenna-to-edge map; any change (other transmitters, reordered receivers,
    other currents) maps again: every S equals a fresh problem's, bit for bit."""
    case = chamber_case(12, 11, n_ant=8)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    tx2 = tx.copy()
    tx2[:, 6:8] *= -1.5
    calls = [(tx, rx), (tx, rx), (tx[:3], rx[::-1]), (tx[:3], rx), (tx2, rx), (tx, rx)]
    P = lib.Problem(M, eps, FREQ, n_sub=4, precision=1, rtol=1e-9)
    got = [P.forward_solve(t, r) for t, r in calls]
    P.close()
    for (t, r), S in zip(calls, got):
        Q = lib.Problem(M, eps, FREQ, n_sub=4, precision=1, rtol=1e-9)
        assert np.array_equal(S, Q.forward_solve(t, r))
        Q.close()
    assert np.array_equal(got[0], got[1]) and np.array_equal(got[0], got[5])
    M.close()


@pytest.mark.parametrize("precision,rtol,tol,max_steps", [(0, 1e-12, 1e-8, 2), (1, 1e-9, 1e-6, 6)])
def test_degenerate_inputs(lib, precision, rtol, tol, max_steps):
    """One transmitter against five receivers (S is 5 x 1); a transmitter with
    zero current among others (its field and S column are exactly zero, and the
    other columns are bit for bit those of the solve without it); one subdomain
    (the ORAS preconditioner is then the factorised operator itself, B_1 = A:
    one or two FGMRES steps in FP64, a few with the FP32 factors)."""
    case = chamber_case(12, 11, n_ant=8)
    mesh, eps, tx, rx, M, topo, perm = _setup(lib, case)
    ref = O.forward(mesh.xyz, topo, eps, FREQ, tx, rx)
    P = lib.Problem(M, eps, FREQ, n_sub=4, precision=precision, rtol=rtol)
    S1 = P.forward_solve(tx[2:3], rx[:5])
    assert S1.shape == (5, 1)
    assert rel_err(S1, ref["S"][:5, 2:3]) <= tol
    assert col_rel_err(P.fields_host(0), ref["U"][perm][:, 2:3]).max() <= tol
    tz = tx.copy()
    tz[3, 6:8] = 0.0
    Sz = P.forward_solve(tz, rx)
    U = P.fields_host(0)
    assert np.all(U[:, 3] == 0) and np.all(Sz[:, 3] == 0)
    keep = [0, 1, 2, 4, 5, 6, 7]
    assert np.array_equal(Sz[:, keep], P.forward_solve(tx[keep], rx))
    P.close()
    P = lib.Problem(M, eps, FREQ, n_sub=1, precision=precision, rtol=rtol)
    S = P.forward_solve(tx, rx)
    info = P.info.as_dict()
    assert info["n_converged"] == 8 and 1 <= info["iters_max"] <= max_steps, info
    assert rel_err(S, ref["S"]) <= tol
    assert col_rel_err(P.fields_host(0), ref["U"][perm]).max() <= tol
    P.close()
    M.close()
