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
    ap.add_argument("--two-level", default="12,11",
                    help="NXY,NZ of the coarse chamber of the two-level ORAS measurement on the main line "
                         "(empty: skip)")
    ap.add_argument("--coarse", default=None,
                    help="with --solve: NXY,NZ of an unjittered coarse chamber whose Whitney space is the coarse "
                         "space of a two-level ORAS")
    ap.add_argument("--nxy", type=int, default=45)
    ap.add_argument("--nz", type=int, default=42)
    ap.add_argument("--n-ant", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nd-leaf", type=int, default=128)
    ap.add_argument("--clocks-csv", default=None, help="directory for the nvidia-smi clock samples (CSV)")
    ap.add_argument("--serve", type=int, default=0,
                    help="run the serving scenario with this many Poisson requests instead of the gradient step")
    ap.add_argument("--serve-requests", type=int, default=100,
                    help="requests of the serving scenario measured after the gradient step (0: skip)")
    ap.add_argument("--serve-freq-step", type=float, default=40e6,
                    help="frequency grid of the serving requests (Hz) in 0.8-1.2 GHz")
    ap.add_argument("--recycle-steps", type=int, default=3,
                    help="timed gradient steps with Krylov recycling across steps (0: skip)")
    ap.add_argument("--block-steps", type=int, default=1,
                    help="timed forward solves comparing true block FGMRES with pseudo-block (0: skip)")
    ap.add_argument("--no-errors", action="store_true",
                    help="skip the accuracy statement (mixed path against the FP64 path at rtol 1e-12)")
    ap.add_argument("--p1-steps", type=int, default=2,
                    help="timed gradient steps with the nodal (P1) parameter (0: skip)")
    ap.add_argument("--engine", type=int, default=0,
                    help="complex FP32 sweep engine (see mwi_solver_opts; 0 = the library default, tcgen05)")
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
        args.two_level = ""
        args.requests = 2
        args.no_cpu_baseline = True
    results["mixed"] = one_arm(1, args.steps, args.warmup, max(2, args.requests))
    if not args.no_errors and not args.only_mixed:
        results["errors"] = error_statement(args, mwi, M, mesh, eps, ants, dev, stream)
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
    # two-level ORAS: one forward solve of the 32 transmitters with the
    # one-level preconditioner and with a coarse space (Whitney elements of an
    # unjittered coarse chamber), at the bench's 64 subdomains and at 1,024
    if args.two_level:
        from synthetic import chamber_mesh
        cxy, cz = [int(v) for v in args.two_level.split(",")]
        cm = chamber_mesh(cxy, cz, jitter=0.0, permute=False)
        Mc = mwi.Mesh(cm.xyz, cm.tet, cm.bface_tag)
        results["two_level"] = {"coarse_grid": [cxy, cz], "runs": []}
        for ns in (64, 1024):
            P = mwi.Problem(M, eps_d, FREQ, stream=stream, n_sub=ns, precision=1, rtol=RTOL, verbose=2,
                            max_iter=500, nd_leaf=args.nd_leaf, sweep_engine=args.engine)
            for coarse in (False, True):
                if coarse:
                    P.set_coarse_space(Mc)
                P.forward_solve(ants, ants)
                P.kernel_times(reset=True)
                torch.cuda.synchronize()
                e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                e0.record(stream)
                P.forward_solve(ants, ants)
                e1.record(stream)
                torch.cuda.synchronize()
                kms, kcnt = P.kernel_times(reset=True)
                info = P.info.as_dict()
                run = {"n_sub": ns, "coarse": coarse, "iterations": info["iters_max"],
                       "forward_ms": round(e0.elapsed_time(e1), 2), "converged": info["n_converged"],
                       "oras_apply_ms": round(float(kms[1]) / max(1, int(kcnt[1])), 3)}
                if coarse:
                    ci = P.coarse_info()
                    run.update(n_coarse=ci["n_coarse"], coarse_setup_ms=round(ci["setup_ms"], 1))
                results["two_level"]["runs"].append(run)
            P.close()
        Mc.close()
    return mesh, M, results


# DRAM bytes of one ORAS apply of the bench workload, summed over its launches
# from ncu's dram__bytes_read.sum + dram__bytes_write.sum (tcgen05 sweeps,
# nested-dissection leaf 128)
ORAS_TRAFFIC = {"bytes_per_call": 8.034e9,
                "source": "ncu DRAM counters of one apply at the bench size, profiles/oras_apply_chamber402k_traffic.md"}


def db_bins(S, S_ref, edges=(0.0, -20.0, -60.0)):
    """Largest entrywise relative error of S against S_ref in bins of
    |S_ref| in dB below its largest entry: [0, -20), [-20, -60), below -60."""
    a = np.abs(S_ref)
    db = 20.0 * np.log10(np.maximum(a, 1e-300) / a.max())
    rel = np.abs(S - S_ref) / np.maximum(a, 1e-300)
    out = {}
    for hi, lo in zip(edges, list(edges[1:]) + [-np.inf]):
        sel = (db <= hi) & (db > lo)
        name = f"{hi:g}..{lo:g} dB"
        out[name] = {"count": int(sel.sum()), "max_rel": float(rel[sel].max()) if sel.any() else None}
    out["lowest_db"] = float(db.min())
    return out


def error_statement(args, mwi, M, mesh, eps, ants, dev, stream):
    """Accuracy of the headline (mixed path, rtol 1e-6) on the bench workload,
    against the plain FP64 path solved to rtol 1e-12 on the same GPU and the
    same inputs (the FP64 path matches the CPU oracle to 1e-8 in the parity
    tests): forward and adjoint fields per column, S per dB bin, J and the
    per-tet gradient."""
    import torch

    from synthetic import add_noise, chamber_target_eps
    target = torch.from_numpy(chamber_target_eps(mesh.xyz, mesh.tet)).to(dev)
    eps0 = torch.from_numpy(eps).to(dev)
    res = {}
    S_meas = None
    for name, prec, rtol in (("ref", 0, 1e-12), ("mixed", 1, RTOL)):
        P = mwi.Problem(M, target, FREQ, stream=stream, n_sub=64, precision=prec, rtol=rtol, max_iter=2000,
                        nd_leaf=args.nd_leaf, sweep_engine=args.engine)
        if S_meas is None:
            S_meas = add_noise(P.forward_solve(ants, ants), eta=0.01, seed=1234)
        P.update_eps(eps0)
        S = P.forward_solve(ants, ants)
        it_f = P.info.iters_max
        J, grad = P.misfit_and_gradient(S_meas)
        res[name] = dict(S=S, J=J, grad=grad, U=P.fields_host(0), L=P.fields_host(1), its=(it_f, P.info.iters_max))
        P.close()
    r, m_ = res["ref"], res["mixed"]
    cu = np.linalg.norm(m_["U"] - r["U"], axis=0) / np.linalg.norm(r["U"], axis=0)
    cl = np.linalg.norm(m_["L"] - r["L"], axis=0) / np.linalg.norm(r["L"], axis=0)
    g_ref = np.abs(r["grad"]).max()
    return {"reference": "plain FP64 GPU path at rtol 1e-12, same inputs (gel + head + inclusion eps_r, S_meas "
                         "from the two-inclusion target with 1 % noise)",
            "rtol": RTOL, "iterations_mixed": m_["its"], "iterations_reference": r["its"],
            "fields_col_rel_max": float(cu.max()), "fields_col_rel_median": float(np.median(cu)),
            "adjoint_col_rel_max": float(cl.max()),
            "S_normwise_rel": float(np.linalg.norm(m_["S"] - r["S"]) / np.linalg.norm(r["S"])),
            "S_by_db_bin": db_bins(m_["S"], r["S"]),
            "J_rel": float(abs(m_["J"] - r["J"]) / abs(r["J"])),
            "grad_normwise_rel": float(np.linalg.norm(m_["grad"] - r["grad"]) / np.linalg.norm(r["grad"])),
            "grad_entry_max_over_max": float(np.abs(m_["grad"] - r["grad"]).max() / g_ref)}


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
# Iterations per column of the oracle's FGMRES + ORAS (exact subdomain solves)
# on the bench workload at rtol 1e-6: a complete oracle run of that workload
# (all 64 subdomains factored, two transmitter columns solved) took 12 for
# both columns.  The timed samples below use it to extrapolate a column.
ORACLE_ITERATIONS = 12


class _SubdomainPool:
    """The oracle's one-level ORAS pieces (oracle.dd: local matrix B_i and its
    SuperLU factors) for a sample of the subdomains, one per forked worker
    process, each timing its own factorisation and its local solve
    y += D_i B_i^-1 R_i x.  Fork only: create it before any CUDA call."""

    def __init__(self, mesh, topo, dec, eps, K, M, ids):
        import multiprocessing as mp
        ctx = mp.get_context("fork")
        self.pipes, self.procs = [], []
        for i in ids:
            a, b = ctx.Pipe()
            p = ctx.Process(target=_SubdomainPool._worker, args=(b, int(i), mesh, topo, dec, eps, K, M))
            p.start()
            self.pipes.append(a)
            self.procs.append(p)
        self.t_factor = [c.recv() for c in self.pipes]

    @staticmethod
    def _worker(conn, i, mesh, topo, dec, eps, K, M):
        import types

        import scipy.sparse.linalg as spla

        import oracle as O
        t0 = time.perf_counter()
        view = types.SimpleNamespace(nsub=1, Td=[dec.Td[i]], R=[dec.R[i]])
        B = O.dd.local_matrices(mesh.xyz, topo, view, eps, FREQ, K, M)[0]
        lu = spla.splu(B.tocsc(), permc_spec="MMD_AT_PLUS_A")
        conn.send(time.perf_counter() - t0)
        rng = np.random.default_rng(i)
        x = rng.standard_normal(topo.ndof) + 1j * rng.standard_normal(topo.ndof)
        y = np.zeros(topo.ndof, dtype=np.complex128)
        while conn.recv():
            t0 = time.perf_counter()
            Ri = dec.R[i]
            y[Ri] += dec.D[i] * lu.solve(np.ascontiguousarray(x[Ri]))
            conn.send(time.perf_counter() - t0)

    def solve_times(self):
        for c in self.pipes:
            c.send(True)
        return [c.recv() for c in self.pipes]

    def close(self):
        for c in self.pipes:
            c.send(False)
        for p in self.procs:
            p.join(timeout=30)


def cpu_oracle_setup(args):
    """The oracle on the bench's own workload: topology, element integrals and
    the assembly of A (single-threaded, as the oracle stands; timed, it is
    part of every gradient step), the decomposition (RCB, 64 subdomains,
    delta = 1), and one sampled subdomain per host core factored in a
    process pool (timed)."""
    import oracle as O
    from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas
    mesh = chamber_mesh(args.nxy, args.nz)
    eps = chamber_eps(mesh.xyz, mesh.tet)
    ants = antenna_array(ring_antennas(args.n_ant))
    topo = O.build_topology(mesh.tet, mesh.bface_tag, mesh.nv, 1)
    K, M = O.element_matrices(mesh.xyz, topo)
    t0 = time.perf_counter()
    A = O.assemble_system(mesh.xyz, topo, eps, FREQ, K=K, M=M)
    t_asm = time.perf_counter() - t0
    nsub = 64
    part = O.dd.rcb_partition(mesh.xyz, mesh.tet, nsub)
    dec = O.dd.Decomposition(mesh.xyz, mesh.tet, topo, part, 1)
    cores = len(os.sched_getaffinity(0))
    ids = np.unique(np.linspace(0, nsub - 1, min(cores, nsub)).round().astype(int))
    pool = _SubdomainPool(mesh, topo, dec, eps, K, M, ids)
    return dict(mesh=mesh, eps=eps, ants=ants, topo=topo, A=A, K=K, M=M, pool=pool, cores=cores, nsub=nsub,
                ids=ids, t_asm=t_asm, t_factor=pool.t_factor)


def cpu_oracle_sample(ctx):
    """One bounded sample of a gradient step: every sampled subdomain's local
    solve (in parallel), one SpMM with the oracle's A, and the dot product +
    update pair of the oracle's Gram-Schmidt, each timed; returns the step
    time extrapolated to 64 subdomains over all cores, ORACLE_ITERATIONS
    iterations per column and 2 x n_ant columns, and its parts."""
    import oracle as O
    topo, A = ctx["topo"], ctx["A"]
    n = topo.ndof
    rng = np.random.default_rng(1)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    t_solve = float(np.mean(ctx["pool"].solve_times()))
    t0 = time.perf_counter()
    for _ in range(3):
        y = A @ x
    t_spmm = (time.perf_counter() - t0) / 3
    t0 = time.perf_counter()
    for _ in range(10):
        h = np.vdot(x, y)
        y = y - h * x
    t_gs = (time.perf_counter() - t0) / 10
    # the main process's share of one pooled apply: the input copied into
    # shared memory and the workers' partial results summed
    parts = np.zeros((ctx["cores"], n), dtype=np.complex128)
    t0 = time.perf_counter()
    z = x.copy()
    for w in range(1, ctx["cores"]):
        z += parts[w]
    t_comb = time.perf_counter() - t0
    per_worker = ctx["nsub"] / ctx["cores"]            # subdomains per process in a full pool
    t_apply = per_worker * t_solve + t_comb
    it = ORACLE_ITERATIONS
    t_col = it * (t_apply + t_spmm) + t_spmm + 0.5 * it * (it + 1) * t_gs
    t_fact = per_worker * float(np.mean(ctx["t_factor"]))
    n_cols = 2 * ctx["ants"].shape[0]
    if "t_grad" not in ctx:
        U = rng.standard_normal((n, n_cols // 2)) + 0j
        t0 = time.perf_counter()
        O.gradient(ctx["mesh"].xyz, topo, ctx["eps"], FREQ, U, U, M=ctx["M"])
        ctx["t_grad"] = time.perf_counter() - t0
    step = ctx["t_asm"] + t_fact + n_cols * t_col + ctx["t_grad"]
    return dict(step=step, value=n_cols / step, t_col=t_col, t_apply=t_apply, t_spmm=t_spmm, t_fact=t_fact,
                t_solve=t_solve)


def cpu_sample_text(ctx, smp):
    return (f"oracle (complex128) on the bench workload ({ctx['mesh'].nt} tets, {ctx['topo'].ndof} DOF, "
            f"{ctx['nsub']} subdomains, {ctx['ants'].shape[0]} + {ctx['ants'].shape[0]} columns): assembly of A "
            f"{ctx['t_asm']:.1f} s (1 thread); {len(ctx['ids'])} of the {ctx['nsub']} subdomains factored (SuperLU) "
            f"and solved, one per process, extrapolated to all subdomains over {ctx['cores']} processes "
            f"(factorisation {smp['t_fact']:.1f} s, ORAS apply {smp['t_apply']:.3f} s); SpMM {smp['t_spmm']:.3f} s; "
            f"{ORACLE_ITERATIONS} FGMRES iterations per column (a complete oracle run of this workload) -> "
            f"{smp['t_col']:.2f} s per column; gradient {ctx['t_grad']:.1f} s; one step = {smp['step']:.0f} s")


def cpu_baseline(args):
    """The oracle as it stands on the bench's own workload over all host cores
    (a bounded, timed sample extrapolated to the whole gradient step)."""
    ctx = cpu_oracle_setup(args)
    try:
        smp = cpu_oracle_sample(ctx)
    finally:
        ctx["pool"].close()
    return {"value": smp["value"], "unit": UNIT, "cores": ctx["cores"], "kind": "oracle",
            "config": "same workload as config.workload", "sample": cpu_sample_text(ctx, smp),
            "s_per_step": round(smp["step"], 1)}


def serving_setup(specs):
    """Meshes of the serving scenario and the request executor: a forward batch
    solves the columns of all its requests at once and hands every request the
    S block of its own antennas; a gradient request adds the adjoint solve and
    the gradient against measurements made from its forward S with 5 % seeded
    noise.  Every problem gets its own CUDA stream."""
    import torch

    from paper_1607_02573_gb300 import mwi
    from synthetic import antenna_array, chamber_eps, chamber_mesh, ring_antennas
    meshes = {}
    for name, (nxy, nz, order, nsub) in specs.items():
        m = chamber_mesh(nxy, nz)
        meshes[name] = (mwi.Mesh(m.xyz, m.tet, m.bface_tag, order=order), chamber_eps(m.xyz, m.tet), nsub, m.nt)
    rings = [antenna_array(ring_antennas(32, z=z)) for z in (0.06, 0.10, 0.14, 0.18, 0.22)]
    opts = dict(precision=1, rtol=RTOL, max_iter=500, max_block=32)

    def make(key):
        M, eps, nsub, _ = meshes[key[0]]
        return mwi.Problem(M, eps, key[1], stream=torch.cuda.Stream(), n_sub=nsub, **opts)

    def estimate(key):
        M, _, nsub, _ = meshes[key[0]]
        return M.estimate_bytes(160, n_sub=nsub, **opts)

    def ants_of(r):
        return np.concatenate([rings[(i + r.seed) % 5] for i in range(r.n_rhs // 32)])

    def run_batch(P, batch):
        out = {}
        if batch[0].kind == "forward":
            sets = [ants_of(r) for r in batch]
            tx = np.concatenate(sets)
            S = P.forward_solve(tx, tx)
            off = 0
            for r, a in zip(batch, sets):
                out[r.rid] = (r.n_rhs, S[off:off + len(a), off:off + len(a)].copy())
                off += len(a)
            return out
        r = batch[0]
        tx = ants_of(r)
        S = P.forward_solve(tx, tx)
        rng = np.random.default_rng(r.seed)
        noise = rng.standard_normal(S.shape) + 1j * rng.standard_normal(S.shape)
        J, grad = P.misfit_and_gradient(S * (1 + 0.05 * noise / np.sqrt(2)))
        out[r.rid] = (2 * r.n_rhs, (S, J, grad))
        return out

    return meshes, make, estimate, run_batch


def run_serving(args, n_requests=None):
    """Serving scenario: Poisson arrivals in real time of imaging requests on
    three resident chamber meshes (about 50k tets at order 2, 200k and 500k
    tets at order 1), 32-160 transmitters in rings of 32, frequencies on a
    grid of 0.8-1.2 GHz (40 MHz by default), forward or misfit+gradient;
    continuous batching over 3 slots (own streams), forward requests of one
    problem merged up to 160 columns, problems cached per (mesh, frequency)
    under a 150 GB budget.  The arrival rate is 70 % of the server's capacity
    measured on a burst of calibration requests.  Returns the summary dict."""
    import torch

    from paper_1607_02573_gb300 import serve as SV

    torch.cuda.set_device(0)
    n_requests = n_requests or args.serve
    specs = {"chamber50k_o2": (23, 21, 2, 16), "chamber200k_o1": (36, 34, 1, 64), "chamber500k_o1": (48, 45, 1, 64)}
    meshes, make, estimate, run_batch = serving_setup(specs)
    budget = 150 * 10 ** 9
    names = list(specs)
    step = args.serve_freq_step
    close = lambda P: P.close()  # noqa: E731
    # calibration: a burst of sample requests through the same server gives its
    # capacity in columns per second; the measured run arrives at 70 % of it
    cal = SV.make_requests(max(12, n_requests // 5), rate=1e6, meshes=names, seed=98, freq_step=step)
    cache = SV.ProblemCache(budget, make, SV.device_bytes, close, estimate=estimate)
    srv = SV.Server(cache, run_batch, slots=3, merge=True, max_cols=160)
    cal_summ = SV.replay(cal, srv)
    cache.clear()
    mean_cols = float(np.mean([r.n_rhs * (2 if r.kind == "gradient" else 1) for r in cal]))
    rate = 0.7 * cal_summ["rhs_solves_per_s"] / mean_cols
    reqs = SV.make_requests(n_requests, rate=rate, meshes=names, seed=99, freq_step=step)
    cache = SV.ProblemCache(budget, make, SV.device_bytes, close, estimate=estimate)
    srv = SV.Server(cache, run_batch, slots=3, merge=True, max_cols=160)
    summ = SV.replay(reqs, srv)
    peak = max(cache.seen.values()) if cache.seen else 0
    cache.clear()
    for M, _, _, _ in meshes.values():
        M.close()
    done = [x for x in srv.records.values() if x["status"] == "done"]
    return dict(summ, arrival_rate_per_s=round(rate, 3), largest_problem_bytes=int(peak), budget_bytes=budget,
                service_s_p50=float(np.percentile([x["service"] for x in done], 50)),
                service_s_p99=float(np.percentile([x["service"] for x in done], 99)),
                calibration_capacity_rhs_per_s=float(cal_summ["rhs_solves_per_s"]),
                meshes={k: {"tets": v[3], "order": specs[k][2], "n_sub": specs[k][3]} for k, v in meshes.items()},
                freq_step_hz=step, slots=3, max_cols=160, rtol=RTOL)


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
                    sweep_engine=args.engine, nd_leaf=args.nd_leaf, verbose=2)
    coarse = None
    if args.coarse:
        cxy, cz = [int(v) for v in args.coarse.split(",")]
        cm = chamber_mesh(cxy, cz, jitter=0.0, permute=False)
        Mc = mwi.Mesh(cm.xyz, cm.tet, cm.bface_tag)
        P.set_coarse_space(Mc)
        Mc.close()
        coarse = dict(P.coarse_info(), grid=[cxy, cz])
        P.kernel_times(reset=True)
    t2 = time.time()
    S = P.forward_solve(ants, ants, allow_notconv=True)
    torch.cuda.synchronize()
    t3 = time.time()
    kms, kcnt = P.kernel_times(reset=True)
    info = P.info.as_dict()
    line = {"mode": "solve", "tets": int(mesh.nt), "dof": int(M.ndof), "order": order, "columns": int(ants.shape[0]),
            "n_sub": n_sub, "precision": prec, "engine": args.engine, "nd_leaf": args.nd_leaf, "mesh_s": round(t1 - t0, 2),
            "setup_s": round(t2 - t1, 2), "forward_s": round(t3 - t2, 3),
            "rhs_solves_per_s": round(ants.shape[0] / (t3 - t2), 2), "factor": P.factor_stats(),
            "oras_impl_bytes_per_call": P.oras_traffic(min(32, ants.shape[0])), "solve": info,
            "kernel_ms": dict(zip(["spmm", "oras_apply", "orthogonalisation", "factorisation"],
                                  [round(v, 2) for v in kms.tolist()])),
            "kernel_calls": kcnt.tolist(), "levels": P.sweep_levels(), "coarse": coarse,
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
        # the oracle on the same workload: assembly and the sampled subdomain
        # factorisations once, then every step a bounded timed sample
        # (cpu_oracle_sample), extrapolated to the whole gradient step
        ctx = cpu_oracle_setup(args)
        n_cols = 2 * args.n_ant
        vals, smp = [], None
        try:
            for k in range(args.warmup + args.steps):
                smp = cpu_oracle_sample(ctx)
                if k >= args.warmup:
                    vals.append(smp["value"])
        finally:
            ctx["pool"].close()
        v = float(np.mean(vals))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": n_cols / v * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
                "data": "synthetic",
                "config": {"workload": workload_name(ctx["mesh"].nt, ctx["topo"].ndof, args)},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": ctx["cores"], "kind": "oracle",
                                 "sample": cpu_sample_text(ctx, smp)},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.serve > 0:
        if rank == 0:
            summ = run_serving(args)
            print(json.dumps({"metric": "serving: latency and RHS-solves/s under Poisson arrivals", "unit": UNIT,
                              "value": round(summ["rhs_solves_per_s"], 3), "higher_is_better": True, "n_gpus": 1,
                              "data": "synthetic", "dtype": "c64+df64", **summ}))
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
        "roofline": roofline(mx, M.ndof, m, traffic=ORAS_TRAFFIC if args.engine in (0, 4) else None),
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
                      if R.get("reuse") else None,
                      "two_level_oras": dict(R["two_level"], what=(
                          "one forward solve of the 32 transmitters (mixed path, rtol 1e-6) with the one-level "
                          "ORAS and with the deflated two-level ORAS, the coarse space being the Whitney "
                          "elements of an unjittered coarse chamber; oras_apply_ms includes the coarse "
                          "correction")) if R.get("two_level") else None},
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
    if R.get("errors"):
        line["errors"] = R["errors"]
    if args.serve_requests > 0 and not args.only_mixed and world == 1:
        summ = run_serving(args, args.serve_requests)
        line["serving"] = {k: (float(f"{v:.4g}") if isinstance(v, float) else v) for k, v in summ.items()}
        line["serving"]["what"] = ("Poisson arrivals in real time, latency from arrival to results on the host; "
                                   "continuous batching over 3 slots with own streams, forward requests of one "
                                   "problem merged, problem cache under a 150 GB budget")
    if cpu_line:
        line["cpu_baseline"] = cpu_line
    print(json.dumps(line))


if __name__ == "__main__":
    main()
