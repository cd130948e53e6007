"""Pins for the oracle's block flexible GMRES (block methods of Section 7,
compared with the pseudo-block GMRES of Section 6.3).

* after k steps each column's residual is the least residual over the block
  Krylov space M K_k(A M, R_0), built explicitly and minimised by a separate
  least-squares solve, and the returned iterate attains it;
* no column ends a step with a larger residual than single-vector GMRES over
  its own space M K_k(A M, r_0c) (that space is contained in the block one);
* once k m reaches n the space is everything and the solve is exact;
* on the chamber system with the ORAS preconditioner, the block solve reaches
  the direct solution in no more steps than the column-by-column FGMRES;
* the initial guess from a recycled subspace (Section 7's recycling) leaves a
  residual orthogonal to A span(Xprev), no other element of the span does
  better, and recycling the exact solutions gives them back.
"""

import numpy as np

import oracle as O
from oracle import block_gmres as bg
from oracle import dd
from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas

FREQ = 1e9


def _system(n, m, seed):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    B = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    P = np.eye(n) + 0.2 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    return A, B, P


def test_iterate_is_least_residual_over_block_space():
    A, B, P = _system(60, 3, 1)
    for k in (1, 2, 4):
        X, hist, steps = bg.block_fgmres(A, B, P, steps=k)
        assert steps == k
        basis = bg.krylov_basis(A, P, B, k, block=True)
        ref = bg.least_residual(A, B, basis)
        got = np.linalg.norm(B - A @ X, axis=0)
        assert np.allclose(got, ref, rtol=1e-8, atol=1e-12 * np.linalg.norm(B))
        assert np.allclose(hist[-1], got, rtol=1e-8, atol=1e-12 * np.linalg.norm(B))


def test_no_column_worse_than_single_vector_gmres():
    A, B, P = _system(80, 4, 2)
    for k in (1, 3, 5):
        X, _, _ = bg.block_fgmres(A, B, P, steps=k)
        got = np.linalg.norm(B - A @ X, axis=0)
        singles = bg.krylov_basis(A, P, B, k, block=False)
        for c in range(B.shape[1]):
            single = bg.least_residual(A, B[:, c:c + 1], singles[c])[0]
            assert got[c] <= single * (1 + 1e-10) + 1e-12


def test_exact_once_space_is_full():
    A, B, P = _system(12, 3, 3)
    X, hist, _ = bg.block_fgmres(A, B, P, steps=4)
    assert np.linalg.norm(B - A @ X) <= 1e-10 * np.linalg.norm(B)
    assert np.allclose(X, np.linalg.solve(A, B), rtol=0, atol=1e-9 * np.abs(np.linalg.solve(A, B)).max())


def test_chamber_with_oras_reaches_direct_solution():
    mesh = chamber_mesh(10, 9)
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ).tocsr()
    part = dd.rcb_partition(mesh.xyz, mesh.tet, 4)
    dec = dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    oras = dd.ORAS(dec, dd.local_matrices(mesh.xyz, topo, dec, eps, FREQ))
    tx = antenna_array(ring_antennas(4, radius=0.08))
    d, s = O.antenna_edges(mesh.xyz, topo, tx)
    B = O.build_rhs(topo.ndof, d, s, tx[:, 6] + 1j * tx[:, 7], FREQ)
    U = O.direct_solve(A, B)[0]
    X, hist, steps = bg.block_fgmres(A, B, oras.apply, steps=60, rtol=1e-10)
    assert np.linalg.norm(U - X, axis=0).max() <= 1e-8 * np.linalg.norm(U, axis=0).min()
    singles = [dd.fgmres(A, B[:, c], oras.apply, rtol=1e-10)[1] for c in range(B.shape[1])]
    assert steps <= max(singles)


def test_recycled_initial_guess_is_least_residual_in_span():
    A, B, P = _system(50, 4, 4)
    rng = np.random.default_rng(5)
    Xprev = np.linalg.solve(A + 0.05 * np.eye(50), B) + 0.01 * rng.standard_normal((50, 4))
    x0 = bg.recycled_initial_guess(A, B, Xprev)
    R = B - A @ x0
    AX = A @ Xprev
    # residual orthogonal to A span(Xprev), so no other element of the span does better
    assert np.abs(AX.conj().T @ R).max() <= 1e-10 * np.abs(AX).max() * np.abs(B).max()
    for _ in range(5):
        other = x0 + Xprev @ (1e-3 * (rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))))
        assert np.all(np.linalg.norm(B - A @ other, axis=0) >= np.linalg.norm(R, axis=0) * (1 - 1e-12))
    # recycling the exact solutions reproduces them
    X = np.linalg.solve(A, B)
    assert np.linalg.norm(bg.recycled_initial_guess(A, B, X) - X) <= 1e-10 * np.linalg.norm(X)
    # a nearby system's solutions already cut the residual
    assert np.linalg.norm(R) < 0.2 * np.linalg.norm(B)
