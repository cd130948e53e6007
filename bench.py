"""Benchmark: RHS-solves/s of the microwave-imaging hot path on one GB300.

One step is one pass of the whole hot path over the 402,444-tet chamber
(radius 0.15 m, height 0.28 m, lowest-order Nedelec, 458,220 DOFs after PEC
removal, 1 GHz, 32 ring antennas, ORAS with 64 subdomains and delta = 1):
re-assemble A and the 64 local operators for eps_r, factorise them as one
batch, solve the 32 state problems, form S and the misfit, solve the 32
adjoint problems with the same factors and reduce the per-tet gradient.  The
mesh topology and the decomposition (partition, overlap, ordering) are built
once before timing, as the paper's setup does per mesh.

value = (32 forward + 32 adjoint columns) x steps / device time, every column
checked to reach a true relative residual <= 1e-6 (residual formed in
double-float, about 48 significant bits).  The mixed path (complex FP32
subdomain factors and ORAS preconditioning an FGMRES whose basis, residual and
iterate are double-float FP32 pairs) is the headline; the plain FP64 path and
the nested variant are measured in the same run.

--impl reference times the CPU oracle (SciPy direct LU, complex128) on a
bounded sample of the same workload family.
"""

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

# The oracle legs spread their work over processes, one per host core; a
# threaded BLAS in every one of them would oversubscribe the cores (set before
# numpy loads its BLAS).  The GPU path does not use BLAS.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS-solves/s @ rel. residual 1e-6, mixed vs plain FP64 GPU; p50/p99 latency"
UNIT = "RHS-solves/s"
FREQ = 1e9
RTOL = 1e-6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--nested-steps", type=int, default=3)
    ap.add_argument("--only-mixed", action="store_true",
                    help="time the mixed arm alone (no other arms, no CPU baseline, 2 e2e requests): for profiling")
    ap.add_argument("--solve", default=None,
                    help="one forward solve instead of the gradient step, for sizing and profiling: "
                         "NXY,NZ,N_SUB,PRECISION[,N_ANT,ORDER,RINGS,MAX_BLOCK,RESTART] "
                         "(defaults 30,28,32,1,32,1,1,64,50: 120,288 tets; RINGS=5 is the 160-antenna layout)")
    ap.add_argument("--nxy", type=int, default=45)
    ap.add_argument("--nz", type=int, default=42)
    ap.add_argument("--n-ant", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nd-leaf", type=int, default=64)
    ap.add_argument("--clocks-csv", default=None, help="directory for the nvidia-smi clock samples (CSV)")
    ap.add_argument("--serve", type=int, default=0,
                    help="run the serving scenario with this many Poisson requests instead of the gradient step")
    ap.add_argument("--serve-freq-step", type=float, default=10e6,
                    help="frequency grid of the serving requests (Hz) in 0.8-1.2 GHz")
    ap.add_argument("--recycle-steps", type=int, default=3,
                    help="timed gradient steps with Krylov recycling across steps (0: skip)")
    ap.add_argument("--block-steps", type=int, default=1,
                    help="timed forward solves comparing true block FGMRES with pseudo-block (0: skip)")
    ap.add_argument("--p1-steps", type=int, default=2,
                    help="timed gradient steps with the nodal (P1) parameter (0: skip)")
    ap.add_argument("--engine", type=int, default=2, help="complex FP32 sweep engine (see mwi_solver_opts)")
    ap.add_argument("--requests", type=int, default=200,
                    help="end-to-end gradient requests (host in, host out) for e2e throughput and p50/p99 latency")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
CLOCK_Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    # samples go to a CSV beside the run (--clocks-csv DIR) or to the temp directory
    out_dir = None

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join(ClockSampler.out_dir or tempfile.gettempdir(), f"mwi_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = np.array([r[0] for r in rows])
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[2]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][1]), "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------- workload
def workload(args):
    from synthetic import (add_noise, antenna_array, chamber_eps, chamber_mesh, chamber_target_eps,
                           ring_antennas)
    mesh = chamber_mesh(args.nxy, args.nz)
    eps0 = np.full(mesh.nt, 44 - 20j)  # homogeneous gel: the inversion's starting point
    eps = chamber_eps(mesh.xyz, mesh.tet)
    ants = antenna_array(ring_antennas(args.n_ant))
    return mesh, eps0, eps, ants


def run_mine(args, rank, world):
    import torch

    from paper_1607_02573_gb300 import mwi

    dev = torch.device("cuda", rank % torch.cuda.device_count())
    torch.cuda.set_device(dev)
    mesh, eps0, eps, ants = workload(args)
    stream = torch.cuda.Stream()
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag, order=1)
    eps_d = torch.from_numpy(eps).to(dev)
    results = {}

    def one_arm(precision, steps, warmup, e2e_steps, recycle=0, factor_reuse=0):
        P = mwi.Problem(M, eps_d, FREQ, stream=stream, n_sub=64, precision=precision, rtol=RTOL,
                        verbose=2, max_iter=500, nd_leaf=args.nd_leaf, sweep_engine=args.engine, recycle=recycle,
                        factor_reuse=factor_reuse)
        fs = P.factor_stats()
        fs["oras_bytes_per_call"] = P.oras_traffic(min(32, args.n_ant))
        fs["nloc"] = int(P.decomposition(64)[1].sum())
        # synthetic measurements: S of the two-inclusion target map plus 1 % noise
        from synthetic import add_noise, chamber_target_eps
        P.update_eps(torch.from_numpy(chamber_target_eps(mesh.xyz, mesh.tet)).to(dev))
        S_t = P.forward_solve(ants, ants)
        S_meas = add_noise(S_t, eta=0.01, seed=1234)
        S_meas_d = torch.from_numpy(np.ascontiguousarray(S_meas.T)).to(dev)  # column-major [n_rx, n_tx]
        grad_d = torch.empty(mesh.nt, dtype=torch.complex128, device=dev)
        eps_steps = [torch.from_numpy(eps * (1 + 0.01 * k)).to(dev) for k in range(2)]
        conv = []

        def step(k):
            import ctypes as C
            P.update_eps(eps_steps[k % 2])
            S = P.forward_solve(ants, ants)
            i1 = P.info.as_dict()
            J = C.c_double()
            info = mwi.mwi_solve_info()
            mwi.check(mwi.mwi_misfit_and_gradient_device(P.h, C.c_void_p(S_meas_d.data_ptr()), None, C.byref(J),
                                                         C.c_void_p(grad_d.data_ptr()), C.byref(info)))
            conv.append(i1["n_converged"] + info.n_converged)
            return i1, info.as_dict()

        for k in range(warmup):
            step(k)
        P.kernel_times(reset=True)
        conv.clear()
        n0 = mwi.mwi_launch_count()
        results.setdefault("launches_before_timed", int(n0))
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        step_ms = []
        with ClockSampler(dev.index) as clk:
            e0.record(stream)
            for k in range(steps):
                ta = torch.cuda.Event(enable_timing=True)
                tb = torch.cuda.Event(enable_timing=True)
                ta.record(stream)
                i_fwd, i_adj = step(k)
                tb.record(stream)
                tb.synchronize()
                step_ms.append(ta.elapsed_time(tb))
            e1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        launches = mwi.mwi_launch_count() - n0
        ms = e0.elapsed_time(e1)
        kms, kcnt = P.kernel_times(reset=True)
        # end-to-end through the public API with host buffers
        # (one request: eps_r from host memory in; S, J and the gradient in host memory out)
        eps_h = [eps * (1 + 0.01 * k) for k in range(2)]
        req_ms = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            ta = time.perf_counter()
            P.update_eps(eps_h[k % 2])
            P.forward_solve(ants, ants)
            P.misfit_and_gradient(S_meas)
            req_ms.append((time.perf_counter() - ta) * 1e3)
        torch.cuda.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / max(1, e2e_steps)
        n_cols = 2 * ants.shape[0]
        res = dict(ms=ms, steps=steps, ms_per_step=ms / steps, value=n_cols * steps / (ms / 1e3),
                   converged=int(sum(conv)), expected=n_cols * steps, launches=int(launches),
                   kernel_ms=kms.tolist(), kernel_calls=kcnt.tolist(), step_ms=step_ms, clocks=clk.summary(),
                   e2e_ms=e2e_ms, e2e_value=n_cols / (e2e_ms / 1e3), req_ms=req_ms, fwd_info=i_fwd, adj_info=i_adj,
                   factor=fs, n_cols=n_cols)
        P.close()
        return res

    if args.only_mixed:
        args.nested_steps = args.fp64_steps = args.recycle_steps = args.block_steps = args.p1_steps = 0
        args.requests = 2
        args.no_cpu_baseline = True
    results["mixed"] = one_arm(1, args.steps, args.warmup, max(2, args.requests))
    results["nested"] = one_arm(2, args.nested_steps, args.warmup, 0) if args.nested_steps > 0 else None
    results["fp64"] = one_arm(0, args.fp64_steps, args.warmup, 0) if args.fp64_steps > 0 else None
    # Krylov recycling: the same step sequence (eps_r alternating between two maps 1 % apart, as
    # consecutive L-BFGS steps), every solve starting from the previous step's solution span
    results["recycle"] = one_arm(1, args.recycle_steps, args.warmup, 0, recycle=1) if args.recycle_steps > 0 else None
    # and keeping the subdomain factors for two of every three steps (factor_reuse = 2)
    results["reuse"] = (one_arm(1, args.recycle_steps, args.warmup, 0, recycle=1, factor_reuse=2)
                        if args.recycle_steps > 0 else None)
    # true block FGMRES (one Krylov space for the 32 columns) against the
    # pseudo-block FGMRES on the same forward solve of the 32 transmitters
    if args.block_steps > 0:
        results["block"] = {}
        for name, bk in (("pseudo_block", 0), ("block", 1)):
            P = mwi.Problem(M, eps_d, FREQ, stream=stream, n_sub=64, precision=1, rtol=RTOL, verbose=2,
                            max_iter=500, nd_leaf=args.nd_leaf, sweep_engine=args.engine, block_krylov=bk)
            P.forward_solve(ants, ants)
            P.kernel_times(reset=True)
            torch.cuda.synchronize()
            e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
            e0.record(stream)
            for _ in range(args.block_steps):
                P.forward_solve(ants, ants)
            e1.record(stream)
            torch.cuda.synchronize()
            fms = e0.elapsed_time(e1) / args.block_steps
            kms, _ = P.kernel_times(reset=True)
            info = P.info.as_dict()
            results["block"][name] = {
                "iterations": info["iters_max"], "forward_ms": round(fms, 2),
                "rhs_solves_per_s": round(ants.shape[0] / (fms / 1e3), 2), "resid_max": info["resid_max"],
                "converged": info["n_converged"],
                "kernel_ms": {k: round(v / args.block_steps, 2) for k, v in
                              zip(["spmm", "oras_apply", "orthogonalisation"], kms[:3].tolist())}}
            P.close()
    # nodal (P1) parameter with the gradient penalty (kappa varying inside every
    # tet): the same gradient step with the vertex parameter, mixed path
    if args.p1_steps > 0:
        P = mwi.Problem(M, eps_d, FREQ, stream=stream, n_sub=64, precision=1, rtol=RTOL, max_iter=500,
                        nd_leaf=args.nd_leaf, sweep_engine=args.engine)
        with torch.cuda.stream(stream):
            kap = torch.full((mesh.nv,), 44 - 20j, dtype=torch.complex128, device=dev)
            kap += torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, mesh.nv)).to(dev)
        S_meas = P.forward_solve(ants, ants) * 1.01
        w = mwi.normalised_weights(S_meas)

        def p1_step():
            P.update_kappa(kap)
            P.forward_solve(ants, ants)
            return P.misfit_and_gradient_kappa(S_meas, w, 1e-3)

        p1_step()
        torch.cuda.synchronize()
        e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
        e0.record(stream)
        for _ in range(args.p1_steps):
            J, R, _ = p1_step()
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / args.p1_steps
        results["p1"] = {"ms_per_step": pms, "value": 2 * ants.shape[0] / (pms / 1e3), "unit": UNIT,
                         "nv": int(mesh.nv), "steps": args.p1_steps, "J": J, "R": R,
                         "what": "gradient step with the nodal parameter (vertex-weighted mass term, "
                                 "normalised misfit, gradient penalty alpha = 1e-3): update_kappa (P1 masses, "
                                 "assembly, factorisation), forward and adjoint solves, vertex gradient"}
        P.close()
    return mesh, M, results


def roofline(res, ndof, m, traffic=None):
    """ORAS apply (gather, forward and backward multifrontal sweeps, scatter),
    HBM-bound.  Algorithmic bytes per call, each operand moved once: the
    complex FP32 factors (every stored panel entry and D^-1 once) plus the
    input and output vectors, n x m complex FP32 each; achieved = those bytes
    / the measured time per call (CUDA events on the problem's stream around
    every call in the timed region), against the measured copy bandwidth.
    The library's own count of what the sweeps must move (factors once per
    sweep, the local and update vectors of every front: mwi_oras_traffic) is
    reported beside it as frac_impl_traffic."""
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    calls = res["kernel_calls"][1]
    if calls == 0:
        return None
    per_call_ms = res["kernel_ms"][1] / calls
    fac = res["factor"]
    alg = (fac["factor_entries"] + fac["nloc"]) * 8.0 + 2.0 * ndof * m * 8.0
    impl = fac["oras_bytes_per_call"]
    achieved = alg / (per_call_ms / 1e3) / 1e9
    peak = peaks.get("hbm_gbs", 6800.0)
    src = "measured copy bandwidth (hbm_gbs) of MEASURED_PEAKS.json" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    flops = 2.0 * 8.0 * fac["factor_entries"] * m
    out = {"bound": "hbm", "kernel": "ORAS apply (c64 multifrontal forward/backward sweeps, gather, scatter)",
           "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
           "traffic": None, "peak_source": src, "algorithmic_bytes_per_call": alg,
           "what_algorithmic": "c64 factor entries (panels + D^-1) once + x in + y out (n x m c64 each)",
           "impl_bytes_per_call": impl,
           "frac_impl_traffic": round(impl / (per_call_ms / 1e3) / 1e9 / peak, 4),
           "ms_per_call": per_call_ms, "tensor_tflops": round(flops / (per_call_ms / 1e3) / 1e12, 2)}
    if traffic:
        out["traffic"] = traffic["bytes_per_call"]
        out["traffic_source"] = traffic["source"]
        out["traffic_over_algorithmic"] = round(traffic["bytes_per_call"] / alg, 3)
    return out


# ---------------------------------------------------------------- CPU baseline (the oracle)
class _OrasPool:
    """The oracle's one-level ORAS (oracle.dd: local matrices B_i, SuperLU per
    subdomain, y = sum_i R_i^T D_i B_i^-1 R_i x) with its subdomains spread
    over forked worker processes, one contiguous share of subdomains each.
    Vectors travel through shared memory; the main process sums the workers'
    partial results in a fixed order.  Fork only: create it before any CUDA
    call in this process."""

    def __init__(self, mesh, topo, dec, eps, K, M, workers):
        import multiprocessing as mp
        self.n = topo.ndof
        self.W = workers
        ctx = mp.get_context("fork")
        self.x = ctx.RawArray("d", 2 * self.n)
        self.y = ctx.RawArray("d", 2 * self.n * workers)
        self.pipes, self.procs = [], []
        shares = np.array_split(np.arange(dec.nsub), workers)
        for w in range(workers):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_OrasPool._worker, args=(b, w, shares[w], mesh, topo, dec, eps, K, M,
                                                            self.x, self.y, self.n))
            p.start()
            self.pipes.append(a)
            self.procs.append(p)
        self.setup_s = max(c.recv() for c in self.pipes)

    @staticmethod
    def _worker(conn, w, ids, mesh, topo, dec, eps, K, M, xs, ys, n):
        import types

        import scipy.sparse.linalg as spla

        import oracle as O
        t0 = time.perf_counter()
        view = types.SimpleNamespace(nsub=len(ids), Td=[dec.Td[i] for i in ids], R=[dec.R[i] for i in ids])
        Bs = O.dd.local_matrices(mesh.xyz, topo, view, eps, FREQ, K, M)
        lus = [spla.splu(B.tocsc(), permc_spec="MMD_AT_PLUS_A") for B in Bs]
        conn.send(time.perf_counter() - t0)
        x = np.frombuffer(xs, dtype=np.complex128)
        y = np.frombuffer(ys, dtype=np.complex128).reshape(-1, n)[w]
        while conn.recv():
            y[:] = 0.0
            for k, i in enumerate(ids):
                Ri = dec.R[i]
                y[Ri] += dec.D[i] * lus[k].solve(np.ascontiguousarray(x[Ri]))
            conn.send(True)

    def apply(self, r):
        x = np.frombuffer(self.x, dtype=np.complex128)
        x[:] = r
        for c in self.pipes:
            c.send(True)
        for c in self.pipes:
            c.recv()
        parts = np.frombuffer(self.y, dtype=np.complex128).reshape(self.W, self.n)
        z = parts[0].copy()
        for w in range(1, self.W):
            z += parts[w]
        return z

    def close(self):
        for c in self.pipes:
            c.send(False)
        for p in self.procs:
            p.join(timeout=30)


def cpu_oracle_setup(args):
    """The oracle on the bench's own workload: topology, element integrals,
    assembly of A (single-threaded, as the oracle stands), the decomposition
    (RCB, 64 subdomains, delta = 1) and, in a pool over all host cores, the
    local matrices and their SuperLU factors."""
    import oracle as O
    from synthetic import add_noise, antenna_array, chamber_eps, chamber_mesh, ring_antennas  # noqa: F401
    t0 = time.perf_counter()
    mesh = chamber_mesh(args.nxy, args.nz)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    ants = antenna_array(ring_antennas(args.n_ant))
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    t1 = time.perf_counter()
    K, M = O.element_matrices(mesh.xyz, topo)
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ, K=K, M=M)
    t2 = time.perf_counter()
    part = O.dd.rcb_partition(mesh.xyz, mesh.tet, 64)
    dec = O.dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    cores = len(os.sched_getaffinity(0))
    pool = _OrasPool(mesh, topo, dec, eps, K, M, cores)
    t3 = time.perf_counter()
    return dict(mesh=mesh, eps=eps, ants=ants, topo=topo, A=A, K=K, M=M, pool=pool, cores=cores,
                mesh_s=t1 - t0, assemble_s=t2 - t1, local_factor_s=t3 - t2)


def cpu_oracle_columns(ctx, cols):
    """Solve the given transmitter columns with the oracle's FGMRES + ORAS to
    the metric's rtol; returns seconds per column and the iteration counts."""
    import oracle as O
    topo, ants = ctx["topo"], ctx["ants"]
    tdof, tsgn = O.antenna_edges(ctx["mesh"].xyz, topo, ants)
    B = O.build_rhs(topo.ndof, tdof, tsgn, ants[:, 6] + 1j * ants[:, 7], FREQ)
    its = []
    t0 = time.perf_counter()
    for j in cols:
        _, it, _ = O.dd.fgmres(ctx["A"], B[:, j], ctx["pool"].apply, rtol=RTOL, restart=50, maxiter=500)
        its.append(it)
    return (time.perf_counter() - t0) / len(cols), its


def cpu_baseline_value(ctx, t_col, n_cols):
    """RHS-solves/s of one oracle gradient step on the bench workload: the
    numeric setup (assembly of A; local matrices and factors in the pool) plus
    n_cols column solves at the sampled time per column (the per-tet gradient
    is a few einsums, timed on the workload's own sizes)."""
    import oracle as O
    topo = ctx["topo"]
    rng = np.random.default_rng(0)
    m = n_cols // 2
    U = rng.standard_normal((topo.ndof, m)) + 0j
    t0 = time.perf_counter()
    O.gradient(ctx["mesh"].xyz, topo, ctx["eps"], FREQ, U, U, M=ctx["M"])
    t_grad = time.perf_counter() - t0
    step = ctx["assemble_s"] + ctx["local_factor_s"] + n_cols * t_col + t_grad
    return n_cols / step, step, t_grad


def cpu_baseline(args, n_sample=2):
    """The oracle as it stands on the bench's own workload, over all host
    cores (subdomain factorisations and solves in a process pool), with a
    bounded sample of columns solved to the metric's rtol."""
    ctx = cpu_oracle_setup(args)
    try:
        t_col, its = cpu_oracle_columns(ctx, list(range(n_sample)))
        n_cols = 2 * args.n_ant
        v, step, t_grad = cpu_baseline_value(ctx, t_col, n_cols)
    finally:
        ctx["pool"].close()
    return {"value": v, "unit": UNIT, "cores": ctx["cores"], "kind": "oracle",
            "config": "same workload as config.workload",
            "sample": f"oracle (complex128) on the bench workload ({ctx['mesh'].nt} tets, {ctx['topo'].ndof} DOF, "
                      f"64 subdomains): assembly of A {ctx['assemble_s']:.1f} s (1 thread), local matrices + SuperLU "
                      f"factors {ctx['local_factor_s']:.1f} s ({ctx['cores']} processes), then {n_sample} of the "
                      f"{n_cols} columns solved by the oracle's FGMRES + ORAS to rtol {RTOL:g} "
                      f"({t_col:.2f} s per column, iterations {its}), gradient {t_grad:.2f} s; one step "
                      f"extrapolated to {n_cols} columns = {step:.1f} s",
            "setup_s": round(ctx["assemble_s"] + ctx["local_factor_s"], 2), "s_per_column": round(t_col, 3),
            "iterations": its}


def run_serving(args):
    """Serving scenario: Poisson arrivals of imaging requests on three resident
    chamber meshes (about 50k tets at order 2, 200k and 500k tets at order 1),
    32-160 transmitters in rings of 32, frequencies on a 10 MHz grid of
    0.8-1.2 GHz, forward or misfit+gradient, problems cached per (mesh,
    frequency) under a 150 GB budget; arrival rate set to 70 % of the capacity
    measured on a calibration sample.  One JSON line."""
    import torch

    from paper_1607_02573_gb300 import mwi
    from paper_1607_02573_gb300 import serve as SV
    from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas

    torch.cuda.set_device(0)
    specs = {"chamber50k_o2": (23, 21, 2, 16), "chamber200k_o1": (36, 34, 1, 64), "chamber500k_o1": (48, 45, 1, 64)}
    meshes = {}
    for name, (nxy, nz, order, nsub) in specs.items():
        m = chamber_mesh(nxy, nz)
        meshes[name] = (mwi.Mesh(m.xyz, m.tet, m.bface_tag, order=order), chamber_eps(m.xyz, m.tet), nsub, m.nt)
    rings = [antenna_array(ring_antennas(32, z=z)) for z in (0.06, 0.10, 0.14, 0.18, 0.22)]

    def make(key):
        M, eps, nsub, _ = meshes[key[0]]
        return mwi.Problem(M, eps, key[1], n_sub=nsub, precision=1, rtol=RTOL, max_iter=500, max_block=32)

    def run(P, r):
        k = r.n_rhs // 32
        ants = np.concatenate([rings[(i + r.seed) % 5] for i in range(k)])
        S = P.forward_solve(ants, ants)
        if r.kind == "forward":
            return r.n_rhs
        rng = np.random.default_rng(r.seed)
        noise = rng.standard_normal(S.shape) + 1j * rng.standard_normal(S.shape)
        P.misfit_and_gradient(S * (1 + 0.05 * noise / np.sqrt(2)))
        return 2 * r.n_rhs

    budget = 150 * 10 ** 9
    names = list(specs)
    # calibration: median service time of a sample of requests (its own cache,
    # freed afterwards; the median leaves out each mesh's one-time
    # decomposition); the measured run arrives at 70 % of that capacity
    step = args.serve_freq_step
    cal = SV.make_requests(max(6, args.serve // 5), rate=1.0, meshes=names, seed=98, freq_step=step)
    cache = SV.ProblemCache(budget, make, SV.device_bytes, lambda P: P.close())
    cal_recs, _ = SV.serve(cal, cache, run)
    cache.clear()
    rate = 0.7 / float(np.median([x["service"] for x in cal_recs]))
    reqs = SV.make_requests(args.serve, rate=rate, meshes=names, seed=99, freq_step=step)
    cache = SV.ProblemCache(budget, make, SV.device_bytes, lambda P: P.close())
    recs, summ = SV.serve(reqs, cache, run)
    peak = max(cache.seen.values()) if cache.seen else 0
    cache.clear()
    for M, _, _, _ in meshes.values():
        M.close()
    line = {"metric": "serving: latency and RHS-solves/s under Poisson arrivals", "unit": UNIT,
            "value": round(summ["rhs_solves_per_s"], 3), "higher_is_better": True, "n_gpus": 1,
            "latency_p50_s": round(summ["latency_p50_s"], 4), "latency_p99_s": round(summ["latency_p99_s"], 4),
            "requests": summ["requests"], "columns": summ["columns"], "arrival_rate_per_s": round(rate, 3),
            "busy_fraction": round(summ["busy_fraction"], 3), "cache_hits": summ["cache_hits"],
            "cache_misses": summ["cache_misses"], "evictions": summ["evictions"],
            "largest_problem_bytes": int(peak), "budget_bytes": budget,
            "meshes": {k: {"tets": v[3], "order": specs[k][2], "n_sub": specs[k][3]} for k, v in meshes.items()},
            "service_s_p50": round(float(np.percentile([x["service"] for x in recs], 50)), 4),
            "service_s_p99": round(float(np.percentile([x["service"] for x in recs], 99)), 4),
            "freq_step_hz": step, "data": "synthetic", "dtype": "c64+df64", "rtol": RTOL}
    print(json.dumps(line))


def run_solve(args):
    """One forward solve of a chamber (--solve): one JSON line with the sizes,
    the setup and solve times, the solver statistics and S's reciprocity."""
    import torch

    from paper_1607_02573_gb300 import mwi
    from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas

    vals = [int(v) for v in args.solve.split(",")]
    nxy, nz, n_sub, prec, n_ant, order, rings, max_block, restart = (vals + [30, 28, 32, 1, 32, 1, 1, 64, 50][
        len(vals):])[:9]
    torch.cuda.set_device(0)
    t0 = time.time()
    mesh = chamber_mesh(nxy, nz)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    zs = [0.14] if rings == 1 else [0.06, 0.10, 0.14, 0.18, 0.22]
    ants = antenna_array([a for z in zs for a in ring_antennas(n_ant, z=z)])
    M = mwi.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag, order=order)
    t1 = time.time()
    P = mwi.Problem(M, eps, FREQ, n_sub=n_sub, precision=prec, rtol=RTOL, max_block=max_block, restart=restart,
                    sweep_engine=args.engine, verbose=2)
    t2 = time.time()
    S = P.forward_solve(ants, ants, allow_notconv=True)
    torch.cuda.synchronize()
    t3 = time.time()
    kms, kcnt = P.kernel_times(reset=True)
    info = P.info.as_dict()
    line = {"mode": "solve", "tets": int(mesh.nt), "dof": int(M.ndof), "order": order, "columns": int(ants.shape[0]),
            "n_sub": n_sub, "precision": prec, "engine": args.engine, "mesh_s": round(t1 - t0, 2),
            "setup_s": round(t2 - t1, 2), "forward_s": round(t3 - t2, 3),
            "rhs_solves_per_s": round(ants.shape[0] / (t3 - t2), 2), "factor": P.factor_stats(),
            "oras_impl_bytes_per_call": P.oras_traffic(min(32, ants.shape[0])), "solve": info,
            "kernel_ms": dict(zip(["spmm", "oras_apply", "orthogonalisation", "factorisation"],
                                  [round(v, 2) for v in kms.tolist()])),
            "kernel_calls": kcnt.tolist(),
            "reciprocity": float(np.linalg.norm(S - S.T) / np.linalg.norm(S))}
    P.close()
    M.close()
    print(json.dumps(line))


def workload_name(nt, ndof, args):
    return (f"chamber r=0.15 m h=0.28 m, {nt} tets, order 1, {ndof} DOF, 1 GHz, {args.n_ant} Tx x {args.n_ant} Rx, "
            f"ORAS N_S=64 delta=1, rtol 1e-6, gradient step (forward + adjoint)")


def max_over_ranks(value, world, device="cpu"):
    """The largest value over all ranks (a job's time is its slowest rank's);
    every rank gets it.  The process group must be initialised when world > 1."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, n_cols, steps, ms):
    """RHS-solves per second of the whole job: every replica solves n_cols
    columns per step, and the job takes ms for its steps."""
    return world * n_cols * steps / (ms / 1e3)


def main():
    args = parse()
    ClockSampler.out_dir = args.clocks_csv
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        # the oracle on the same workload: numeric setup once, then every step a
        # bounded sample (one transmitter column to rtol), extrapolated to the
        # step's 2 x n_ant columns
        ctx = cpu_oracle_setup(args)
        n_cols = 2 * args.n_ant
        vals, its, cols = [], [], []
        try:
            for k in range(args.warmup + args.steps):
                t_col, it = cpu_oracle_columns(ctx, [k % args.n_ant])
                if k >= args.warmup:
                    vals.append(cpu_baseline_value(ctx, t_col, n_cols)[0])
                    its += it
                    cols.append(t_col)
        finally:
            ctx["pool"].close()
        v = float(np.mean(vals))
        sample = (f"oracle (complex128) on the bench workload: assembly of A {ctx['assemble_s']:.1f} s (1 thread), "
                  f"local matrices + SuperLU factors {ctx['local_factor_s']:.1f} s ({ctx['cores']} processes), "
                  f"measured once; each step solves one transmitter column with the oracle's FGMRES + ORAS to "
                  f"rtol {RTOL:g} ({np.mean(cols):.2f} s per column, iterations {sorted(set(its))}) and "
                  f"extrapolates setup + {n_cols} columns + gradient")
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": n_cols / v * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic",
                "config": {"workload": workload_name(ctx["mesh"].nt, ctx["topo"].ndof, args)},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": ctx["cores"], "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.serve > 0:
        if rank == 0:
            run_serving(args)
        return
    if args.solve:
        if rank == 0:
            run_solve(args)
        return
    # the CPU baseline forks its process pool, so it runs before any CUDA call
    cpu_line = None
    if not args.no_cpu_baseline and not args.only_mixed and world == 1:
        cpu_line = cpu_baseline(args)
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", rank=rank, world_size=world)
    mesh, M, R = run_mine(args, rank, world)
    mx = R["mixed"]
    ms = max_over_ranks(mx["ms"], world, "cuda")
    value = whole_job_value(world, mx["n_cols"], mx["steps"], ms)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    m = 32 if args.n_ant >= 32 else args.n_ant
    nt = mesh.nt
    h2d = nt * 16 + mx["n_cols"] // 2 * mx["n_cols"] // 2 * 16 + 2 * args.n_ant * 64
    d2h = 2 * (args.n_ant * args.n_ant * 16) + nt * 16 + 8
    step_ms = np.array(mx["step_ms"])
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / mx["steps"], 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+df64", "data": "synthetic",
        "config": {"workload": workload_name(nt, M.ndof, args),
                   "step": "assemble+factorise(64 subdomains)+forward(32 cols)+S+misfit+adjoint(32 cols)+gradient",
                   "precision": "mixed: c64 factors and ORAS application preconditioning an FGMRES whose "
                                "basis, residual and iterate are double-float FP32 pairs (df64); Hessenberg, "
                                "least squares and misfit in FP64",
                   "l2": "working set larger than L2 (c64 factors 2.2 GB, Krylov bases > 1 GB) on every step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "latency_ms": {"p50": round(float(np.percentile(mx["req_ms"], 50)), 3),
                       "p99": round(float(np.percentile(mx["req_ms"], 99)), 3), "requests": len(mx["req_ms"]),
                       "what": "per gradient request, host wall clock: eps_r in host memory -> S, J and the "
                               "per-tet gradient in host memory",
                       "device_step_p50": round(float(np.percentile(step_ms, 50)), 3),
                       "device_step_p99": round(float(np.percentile(step_ms, 99)), 3)},
        "converged_columns": mx["converged"], "expected_columns": mx["expected"],
        "gpu_launches": mx["launches"],
        "launches_before_timed": R.get("launches_before_timed"),
        "e2e": {"value": round(mx["e2e_value"] * world, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": mx["clocks"],
        "roofline": roofline(mx, M.ndof, m),
        "kernel_ms_per_step": {k: round(v / mx["steps"], 3) for k, v in
                               zip(["spmm", "oras_apply", "orthogonalisation", "factorisation"], mx["kernel_ms"])},
        "solver": {"fwd": mx["fwd_info"], "adj": mx["adj_info"], "factor": mx["factor"]},
        "next_rows": {"p1_parameter": {k: (round(v, 4) if isinstance(v, float) else v)
                                       for k, v in R["p1"].items()} if R.get("p1") else None,
                      "block_fgmres": dict(R["block"], what="forward solve of the 32 transmitters, FP32 ORAS "
                                           "preconditioner; block: one shared Krylov space, FP64 block vectors; "
                                           "pseudo_block: the double-float per-column FGMRES of the main line")
                      if R.get("block") else None,
                      "krylov_recycling": {
                          "value": round(R["recycle"]["value"], 3), "unit": UNIT,
                          "ms_per_step": round(R["recycle"]["ms_per_step"], 2), "steps": R["recycle"]["steps"],
                          "fwd_iterations": R["recycle"]["fwd_info"]["iters_max"],
                          "adj_iterations": R["recycle"]["adj_info"]["iters_max"],
                          "converged_columns": R["recycle"]["converged"],
                          "expected_columns": R["recycle"]["expected"],
                          "kernel_ms_per_step": {k: round(v / R["recycle"]["steps"], 3) for k, v in
                                                 zip(["spmm", "oras_apply", "orthogonalisation", "factorisation"],
                                                     R["recycle"]["kernel_ms"])},
                          "what": "the main line's gradient steps with recycle = 1: each forward solve starts "
                                  "from the least-residual element of the span of the previous step's forward "
                                  "solutions, each adjoint solve from that of the current forward and the "
                                  "previous adjoint solutions"} if R.get("recycle") else None,
                      "recycling_with_factor_reuse": {
                          "value": round(R["reuse"]["value"], 3), "unit": UNIT,
                          "ms_per_step": round(R["reuse"]["ms_per_step"], 2), "steps": R["reuse"]["steps"],
                          "fwd_iterations": R["reuse"]["fwd_info"]["iters_max"],
                          "adj_iterations": R["reuse"]["adj_info"]["iters_max"],
                          "converged_columns": R["reuse"]["converged"],
                          "expected_columns": R["reuse"]["expected"],
                          "kernel_ms_per_step": {k: round(v / R["reuse"]["steps"], 3) for k, v in
                                                 zip(["spmm", "oras_apply", "orthogonalisation", "factorisation"],
                                                     R["reuse"]["kernel_ms"])},
                          "what": "as krylov_recycling, with factor_reuse = 2: two of every three eps_r updates "
                                  "keep the previous subdomain factors as the preconditioner"}
                      if R.get("reuse") else None},
    }
    if R["fp64"]:
        f = R["fp64"]
        line["fp64"] = {"value": round(f["value"], 3), "ms_per_step": round(f["ms_per_step"], 1),
                        "steps": f["steps"], "converged_columns": f["converged"],
                        "kernel_ms_per_step": {k: round(v / f["steps"], 2) for k, v in
                                               zip(["spmm", "oras_apply", "orthogonalisation", "factorisation"],
                                                   f["kernel_ms"])},
                        "fwd": f["fwd_info"], "adj": f["adj_info"]}
        line["mixed_over_fp64"] = round(value / world / f["value"], 2)
    if R.get("nested"):
        f = R["nested"]
        line["mixed_nested"] = {"value": round(f["value"], 3), "ms_per_step": round(f["ms_per_step"], 1),
                                "steps": f["steps"], "converged_columns": f["converged"],
                                "what": "inner c64 GMRES(ORAS) as flexible preconditioner of the c128 FGMRES",
                                "kernel_ms_per_step": {k: round(v / f["steps"], 2) for k, v in
                                                       zip(["spmm", "oras_apply", "orthogonalisation",
                                                            "factorisation"], f["kernel_ms"])},
                                "fwd": f["fwd_info"], "adj": f["adj_info"]}
    if cpu_line:
        line["cpu_baseline"] = cpu_line
    print(json.dumps(line))


if __name__ == "__main__":
    main()
