"""Continuous batching on the GPU: every request's result is the same alone
and in a mix of overlapping requests.

A burst of forward and gradient requests on two meshes and two frequencies
goes through the server with three slots (batches on different problems
overlap on the device, each problem on its own stream) and merging (queued
forward requests of one problem solved as one block).  Then every request is
run alone on a fresh problem.  The pseudo-block FGMRES keeps every column's
Krylov space separate and every reduction has a fixed order, so S, J and the
gradient must agree bit for bit.
"""

import numpy as np
import pytest

from paper_1607_02573_gb300 import serve as SV
from tests._helpers import FREQ, chamber_case, cube_case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    return mwi


def test_results_alone_and_in_the_mix_agree(lib):
    cases = {"cube": (cube_case(6), 4), "chamber": (chamber_case(12, 11, n_ant=8), 8)}
    meshes = {}
    for name, ((mesh, eps, tx, rx), nsub) in cases.items():
        meshes[name] = (lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag), eps, nsub, tx)
    opts = dict(precision=1, rtol=1e-9, max_iter=400)

    def make(key):
        M, eps, nsub, _ = meshes[key[0]]
        return lib.Problem(M, eps, key[1], stream=torch.cuda.Stream(), n_sub=nsub, **opts)

    def ants_of(r):
        tx = meshes[r.mesh][3]
        rng = np.random.default_rng(r.seed)
        return tx[np.sort(rng.choice(len(tx), r.n_rhs, replace=False))]

    def run_batch(P, batch):
        out = {}
        if batch[0].kind == "forward":
            sets = [ants_of(r) for r in batch]
            a = np.concatenate(sets)
            S = P.forward_solve(a, a)
            off = 0
            for r, s in zip(batch, sets):
                out[r.rid] = (r.n_rhs, S[off:off + len(s), off:off + len(s)].copy())
                off += len(s)
            return out
        r = batch[0]
        a = ants_of(r)
        S = P.forward_solve(a, a)
        J, grad = P.misfit_and_gradient(S * 0.9)
        out[r.rid] = (2 * r.n_rhs, (S, J, grad))
        return out

    rng = np.random.default_rng(7)
    reqs = []
    for i in range(12):
        name = ["cube", "chamber"][rng.integers(2)]
        nmax = len(meshes[name][3])
        reqs.append(SV.Request(rid=i, arrival=0.0, mesh=name, freq=[FREQ, 1.1e9][rng.integers(2)],
                               kind="forward" if rng.random() < 0.6 else "gradient",
                               n_rhs=int(rng.integers(2, nmax + 1)), seed=int(rng.integers(1 << 20))))
    est = lambda key: meshes[key[0]][0].estimate_bytes(64, n_sub=meshes[key[0]][2], **opts)  # noqa: E731
    cache = SV.ProblemCache(40 * 10 ** 9, make, SV.device_bytes, lambda P: P.close(), estimate=est)
    srv = SV.Server(cache, run_batch, slots=3, merge=True, max_cols=64)
    summ = SV.replay(reqs, srv)
    assert summ["done"] == len(reqs), srv.records
    assert summ["merged_requests"] >= 1 and summ["mean_batches_in_flight"] > 1.0, summ
    mix = dict(srv.results)
    # the estimate taken before building bounds what the problems hold
    for key, e in cache.entries.items():
        assert est(key) >= e[1], (key, est(key), e[1])
    cache.clear()
    for r in reqs:
        P = make((r.mesh, r.freq))
        alone = run_batch(P, [r])[r.rid][1]
        P.close()
        if r.kind == "forward":
            assert np.array_equal(alone, mix[r.rid]), r
        else:
            assert np.array_equal(alone[0], mix[r.rid][0]) and alone[1] == mix[r.rid][1], r
            assert np.array_equal(alone[2], mix[r.rid][2]), r
    for M, _, _, _ in meshes.values():
        M.close()
