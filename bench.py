#!/usr/bin/env python3
"""WaveHoltz benchmark: GLUP/s of one WaveHoltz iteration on one GB300.

A step is one WaveHoltz iteration (the hot path: M = Np * Nt time steps of the explicit
scheme on every component grid, ghost rules, overset interpolation, the fused time
filter; Algorithm 1/2) on the disk-in-square overset workload: Cartesian background
[-2, 2]^2 at 1024^2 + stretched annulus 2048 x 64 around r = 0.5 (width 0.3), order 4,
Neumann on the cylinder, Dirichlet on the box, c = 1, omega = 40, one seeded Gaussian
source, 5x5 Lagrange interpolation, FP64.  Steps chain as fixed-point iterations
v <- W_h(v, f).  GLUP = active-point time-step updates.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 runs under torchrun: the single solve does not shard (replicas only), each rank
runs an independent replica (own seed) and value is the total over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "WaveHoltz GLUP/s (one WaveHoltz iteration, FP64, disk-in-square 1024^2+2048x64 o4)"
WORKLOAD = ("disk-in-square overset: background [-2,2]^2 1024^2 + annulus 2048x64 "
            "(r 0.5..0.8, stretched), order 4, Neumann cylinder / Dirichlet box, c=1, "
            "omega=40, 1 seeded Gaussian, 5x5 Lagrange interpolation, Np=1")
L2_BYTES = 129 * 1024 * 1024


def whole_job(lups_local, t_local, world):
    """Whole-job throughput of `world` replicas: the point updates of all ranks divided by
    the slowest rank's time (max over ranks).  Returns (GLUP/s, t_max in s)."""
    import torch
    if world <= 1:
        return lups_local / t_local / 1e9, t_local
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    n = torch.tensor([float(lups_local)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    t_max = float(t.item())
    return float(n.item()) / t_max / 1e9, t_max


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=5.0):
        """Block until the sampler has produced a line (nvidia-smi takes a while to start)."""
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def mark(self):
        return len(self.lines)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, start=0):
        """Samples from index `start` (the timed region's start) on; if none arrived there,
        all samples (warm-up included), flagged by "window"."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines, window = self.lines[start:], "timed"
        if not lines:
            lines, window = self.lines, "warmup+timed"
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


def stage(msg):
    """Progress on stderr (the JSON line stays alone on stdout)."""
    print(f"[bench] {msg}", file=sys.stderr, flush=True)


def kernel_sha():
    p = os.path.join(ROOT, "paper_2504_03074_gb300", "csrc", "wh_kernels.cu")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def recorded_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from profiles/traffic.txt if it was captured
    from the current kernel source (sha match), else None."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    sha = kernel_sha()
    for line in open(p):
        f = line.split("#")[0].split()
        if len(f) == 3 and f[0] == kernel and f[1] == sha:
            return float(f[2])
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return {}


# FP64 peak of a GB300 for the ALU roofline: 1.25 TFLOP/s (FMA = 2 FLOP), the pool's
# stated figure for this part.
FP64_PEAK_TFLOPS = 1.25
# Algorithmic FP64 FLOP per active-point update of the order-4 march with the fused
# filter: 4 additions pairing symmetric neighbours + 7 multiply-adds (5 stencil
# coefficients, the forcing term, the filter) = 4 + 14.
FLOP_PER_LUP_O4 = 18.0


def cpu_baseline(problem, sample):
    """Time the CPU oracle, as it stands, on a bounded sample: single thread, and the same
    source built with OpenMP over its point loops on all host cores (the same arithmetic:
    its result is checked to equal the single-thread one bit for bit).  `value` and `cores`
    are the all-cores figures."""
    import numpy as np
    from oracle import oracle as O
    from paper_2504_03074_gb300 import grids as G
    v = G.random_state(problem, 1)
    orc = O.Oracle(problem)
    t0 = time.perf_counter()
    ref = orc.iterate(v, True)
    dt1 = time.perf_counter() - t0
    lups = problem.n_active * orc.time.M
    rec = {"value": lups / dt1 / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
           "sample": sample, "seconds": dt1, "host": host_cpu(),
           "single_thread": {"value": lups / dt1 / 1e9, "seconds": dt1, "cores": 1}}
    try:
        omp = O.Oracle(problem, openmp=True)
        t0 = time.perf_counter()
        out = omp.iterate(v, True)
        dtn = time.perf_counter() - t0
        threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
        rec.update({"value": lups / dtn / 1e9, "cores": threads, "seconds": dtn,
                    "all_cores": {"value": lups / dtn / 1e9, "seconds": dtn, "cores": threads,
                                  "equals_single_thread": bool(np.array_equal(out, ref))}})
    except Exception as e:  # no OpenMP toolchain on the host: single thread only
        rec["all_cores"] = {"unavailable": str(e)[:200]}
    return rec


def host_cpu():
    """CPU model and logical core count of this host (the oracle uses one core)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        model = None
    return {"model": model, "logical_cores": os.cpu_count()}


def time_iterations(WH, torch, solver, n_total, stream, flush, reps, warm=2):
    """Device time (s) per WaveHoltz iteration, CUDA events on the library's stream, L2
    flushed between iterations."""
    a = torch.zeros(n_total, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    with torch.cuda.stream(stream):
        for _ in range(warm):
            solver.iterate(a, b, True)
            a, b = b, a
        tot = 0.0
        for k in range(reps):
            if flush is not None:  # inputs larger than L2 need no flush
                flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.iterate(a, b, True)
            e1.record(stream)
            a, b = b, a
            stream.synchronize()
            tot += e0.elapsed_time(e1) / 1e3
    return tot / reps


def measure_forms(WH, G, torch, prob, stream, flush, rank, cpu=True):
    """The FP32-march form on the same workload, the differentiation form (S^T and one
    gradient sweep), the 256-instance batch (batched FP32 and FP64 iterations vs plain
    per-instance FP64 iterations on a sample of instances), Helmholtz solves/s to 1e-6
    relative error on a 16-instance batch (batched FP32/FP64 vs plain FP64), and time to
    1e-6 relative error on the 64^2 unit square."""
    out = {}
    s32 = WH.Solver(prob, stream=stream, precision=WH.FP32)
    ti = s32.prepare()
    t32 = time_iterations(WH, torch, s32, prob.n_total, stream, flush, 5)
    stage("forms: fp32_march")
    out["fp32_march"] = {"value": ti.n_active * ti.M / t32 / 1e9, "unit": "GLUP/s",
                         "ms_per_iteration": t32 * 1e3,
                         "workload": "same disk-in-square workload, FP32 march, FP64 filter"}
    s32.close()
    # several bodies: two ellipses (elliptic-coordinate grids) and a disk in a 1024^2
    # background, order 4, omega 40: one iteration in FP64 and with the FP32 march
    ep = G.ellipses_problem(nb=1024, omega=40.0, scale=2)
    rec = {"workload": "two ellipses + a disk in [-2,2]^2: 1024^2 background + 3 body grids "
                       "(%d points), order 4, omega 40" % ep.n_total}
    for name, prec in (("fp64", WH.FP64), ("fp32", WH.FP32)):
        se = WH.Solver(ep, stream=stream, precision=prec)
        te = se.prepare()
        tt = time_iterations(WH, torch, se, ep.n_total, stream, flush, 5)
        rec[name] = {"value": te.n_active * te.M / tt / 1e9, "unit": "GLUP/s",
                     "ms_per_iteration": tt * 1e3, "M": te.M}
        se.close()
    stage("forms: ellipses_1024")
    out["ellipses_1024"] = rec
    # differentiation form: the transposed map S^T (the product of the adjoint GMRES) and
    # one gradient sweep (forward march from u kept whole in HBM, reverse sweep with the
    # c^2 and f gradients); g = 0 makes the adjoint GMRES return at once, so the call times
    # the sweep alone
    sa = WH.Solver(prob, stream=stream)
    ta = sa.prepare()
    n = prob.n_total

    def timed(fn, reps, warm=2):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                fn()
            tot = 0.0
            for k in range(reps):
                flush.fill_(float(k))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                stream.synchronize()
                tot += e0.elapsed_time(e1) / 1e3
        return tot / reps

    def adjoint_costs(sa, ta, n):
        x = torch.randn(n, dtype=torch.float64, device="cuda")
        y = torch.empty_like(x)
        zero = torch.zeros_like(x)
        tf = time_iterations(WH, torch, sa, n, stream, flush, 5)
        tt = timed(lambda: sa.apply_adjoint(x, y), 5)
        tg = timed(lambda: sa.adjoint(x, zero, 1e-8, 10, 10), 3)
        return {"transpose_apply": {"value": ta.n_active * ta.M / tt / 1e9, "unit": "GLUP/s",
                                    "ms": tt * 1e3, "vs_forward_iteration": tt / tf},
                "gradient_sweep": {"ms": tg * 1e3, "vs_forward_iteration": tg / tf},
                "forward_iteration_ms": tf * 1e3}

    stage("forms: adjoint")
    out["adjoint"] = adjoint_costs(sa, ta, n)
    out["adjoint"]["workload"] = "same disk-in-square workload, FP64"
    sa.close()
    # the sound-speed inversion geometry: 512^2 background + 1024x32 annulus, omega 20,
    # c = 1 + 0.2 sum of 8 Gaussian bumps (every grid on per-point weights)
    mp = G.misfit_problem(nb=512, omega=20.0, seed=0)
    sm = WH.Solver(mp, stream=stream)
    tm = sm.prepare()
    stage("forms: adjoint_misfit_512")
    out["adjoint_misfit_512"] = adjoint_costs(sm, tm, mp.n_total)
    out["adjoint_misfit_512"]["workload"] = (
        "disk-in-square 512^2 + 1024x32, order 4, omega 20, c = 1 + 0.2 sum of 8 Gaussian "
        "bumps (width 0.2), FP64; M = %d" % tm.M)
    sm.close()
    # time to the gradient on that geometry: N_p = 4, the reverse march from checkpoints
    # every 16 steps; forward GMRES to 1e-12, the receiver misfit against data from a
    # medium 5% faster in a Gaussian patch, adjoint GMRES to 1e-12 and the gradient sweep
    # (the gradients' agreement with central finite differences is a GPU test)
    stage("forms: gradient_misfit_512_np4")
    P = G.receiver_matrix(mp, n=64, radius=1.5)
    sg = WH.Solver(mp, stream=stream, periods=4, trajectory_bytes=1)
    for gi, c in enumerate(G.perturbed_c2(mp)):
        sg.set_coefficient(gi, c)
    sg.prepare()
    ud, _ = _solve_timed(WH, torch, sg, mp.n_total, 1e-10, 3000, restart=400)
    d = P @ ud.cpu().numpy()
    for gi, c in enumerate(mp.c2):
        sg.set_coefficient(gi, c)
    tg = sg.prepare()
    u, fw = _solve_timed(WH, torch, sg, mp.n_total, 1e-12, 3000, restart=400)
    rr = P @ u.cpu().numpy() - d
    g = torch.from_numpy(P.T @ rr).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, gc2, gf, sta = sg.adjoint(u, g, tol=1e-12, max_it=3000, restart=400)
    torch.cuda.synchronize()
    ta_s = time.perf_counter() - t0
    out["gradient_misfit_512_np4"] = {
        "M": tg.M, "misfit": 0.5 * float(rr @ rr), "forward": fw,
        "adjoint": {"seconds": ta_s, "wave_solves": sta.iterations, "residual": sta.residual,
                    "converged": sta.converged},
        "time_to_gradient_s": fw["seconds"] + ta_s,
        "grad_c2_norm": float(gc2.norm()), "grad_f_norm": float(gf.norm())}
    sg.close()
    del u, ud, gc2, gf, g
    # batch: 256 disk-in-square instances, N ~ U{256..1024}, annulus 2N x N/16,
    # omega ~ U[10, 50], 1-4 sources
    t0 = time.perf_counter()
    bp, probs = G.batch_disk_problem(256, seed=100 + rank)
    gen_s = time.perf_counter() - t0
    res = {"instances": len(probs), "points": bp.n_total,
           "active_points": int(sum(p.n_active for p in probs)), "generate_s": gen_s}
    for name, prec in (("fp32", WH.FP32), ("fp64", WH.FP64)):
        sb = WH.Solver(bp, stream=stream, precision=prec)
        infos = sb.prepare()
        lups = sum(t.n_active * t.M for t in infos)
        tuned = sb.autotune(reps=1)  # launch layout picked by timing each candidate (untimed)
        tb = time_iterations(WH, torch, sb, bp.n_total, stream, flush, 2, warm=1)
        res[f"batched_{name}"] = {"value": lups / tb / 1e9, "unit": "GLUP/s",
                                  "s_per_iteration": tb, "layout": tuned}
        sb.close()
        del sb
    # plain FP64, one instance at a time, on 8 seeded instances (GLUP/s by LUP count)
    rng = __import__("numpy").random.default_rng(7)
    pick = rng.choice(len(probs), size=8, replace=False)
    tl, ll = 0.0, 0
    for k in pick:
        sp = WH.Solver(probs[k], stream=stream)
        tk = sp.prepare()
        tl += time_iterations(WH, torch, sp, probs[k].n_total, stream, flush, 1, warm=1)
        ll += tk.n_active * tk.M
        sp.close()
    res["plain_fp64_per_instance"] = {"value": ll / tl / 1e9, "unit": "GLUP/s",
                                      "sample": "8 seeded instances, one at a time"}
    res["speedup_batched_fp32_vs_plain_fp64"] = res["batched_fp32"]["value"] / \
        res["plain_fp64_per_instance"]["value"]
    stage("forms: batch_256")
    out["batch_256"] = res
    del bp, probs
    # Helmholtz solves/s to 1e-6 relative error: batched FP32 (refined), batched FP64 and
    # plain FP64 one instance at a time, on a seeded batch of 16 smaller, lower-frequency
    # disk-in-square instances (the 256-instance sizes need thousands of wave solves per
    # instance at Np = 1).  Errors against an FP64 batched solve to 1e-13 (untimed).
    sb_p, sb_probs = G.batch_disk_problem(16, seed=11, nb_range=(128, 256),
                                          omega_range=(6.0, 12.0), width=0.6, r_cut=0.7)
    ref = WH.Solver(sb_p, stream=stream)
    ref.prepare()
    uref = torch.zeros(sb_p.n_total, dtype=torch.float64, device="cuda")
    ref.solve_batch(uref, tol=1e-13, max_it=8000, restart=400)
    ref.close()
    offs = [0]
    for q in sb_probs:
        offs.append(offs[-1] + q.n_total)

    def worst_err(u):
        e = 0.0
        for a, b in zip(offs[:-1], offs[1:]):
            r = uref[a:b]
            e = max(e, float((u[a:b] - r).abs().max() / r.abs().max()))
        return e

    tol = 3e-11  # these instances are conditioned near 1e4: residual 3e-11 gives <= 1e-6 error
    bs = {"instances": len(sb_probs), "points": sb_p.n_total, "tol": tol,
          "workload": "16 seeded disk-in-square instances, N ~ U{128..256}, annulus 2N x N/16, "
                      "omega ~ U[6, 12], order 4; solves to relative residual 3e-11"}
    for name, prec in (("batched_fp32", WH.FP32), ("batched_fp64", WH.FP64)):
        sv = WH.Solver(sb_p, stream=stream, precision=prec)
        sv.prepare()
        u = torch.zeros_like(uref)
        sv.solve_batch(u, tol=tol, max_it=8000, restart=400)  # warm-up (graphs)
        u.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sts = sv.solve_batch(u, tol=tol, max_it=8000, restart=400)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        bs[name] = {"solves_per_s": len(sb_probs) / el, "seconds": el,
                    "max_rel_err": worst_err(u), "converged": int(sum(x.converged for x in sts))}
        sv.close()
    el, solved = 0.0, 0
    uu = torch.zeros_like(uref)
    for q, a, b in zip(sb_probs, offs[:-1], offs[1:]):
        sv = WH.Solver(q, stream=stream)
        sv.prepare()
        u = torch.zeros(q.n_total, dtype=torch.float64, device="cuda")
        sv.solve(u, WH.GMRES, tol=tol, max_it=8000, restart=400)  # warm-up (graphs)
        u.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = sv.solve(u, WH.GMRES, tol=tol, max_it=8000, restart=400)
        torch.cuda.synchronize()
        el += time.perf_counter() - t0
        solved += int(st.converged)
        uu[a:b] = u
        sv.close()
    bs["plain_fp64"] = {"solves_per_s": len(sb_probs) / el, "seconds": el,
                        "max_rel_err": worst_err(uu), "converged": solved}
    bs["speedup_batched_fp32_vs_plain_fp64"] = bs["batched_fp32"]["solves_per_s"] / \
        bs["plain_fp64"]["solves_per_s"]
    bs["speedup_batched_fp64_vs_plain_fp64"] = bs["batched_fp64"]["solves_per_s"] / \
        bs["plain_fp64"]["solves_per_s"]
    stage("forms: batch_solve")
    out["batch_solve"] = bs
    del sb_p, sb_probs, uref
    # roofline probe: one Cartesian grid of 16384^2 points (HBM resident), no interpolation,
    # orders 2 and 4, FP64 and FP32; the march kernel's device time per launch from a
    # graph-captured burst (an iteration would be ~11,600 steps here).  Effective bandwidth
    # counts the compulsory bytes of one update (48 B FP64, 32 B FP32 state + FP64 filter).
    hbm = float(measured_peaks().get("hbm_gbs", 6793.0))
    probe = {"workload": "unit square 16384^2, Dirichlet, omega 10, no interpolation",
             "hbm_peak_gbs": hbm}
    for order in (2, 4):
        pp = G.unit_square_problem(16384, order, 10.0, seed=0)
        for name, prec, bpl in (("fp64", WH.FP64, 48.0), ("fp32", WH.FP32, 32.0)):
            sp = WH.Solver(pp, stream=stream, precision=prec)
            tp = sp.prepare()
            ms = sp.profile_kernels(reps=10)["march"][0]
            glups = tp.n_active / (ms * 1e-3) / 1e9
            rec = {"march_us": ms * 1e3, "value": glups, "unit": "GLUP/s",
                   "effective_gbs": glups * bpl, "hbm_frac": glups * bpl / hbm}
            if prec == WH.FP64:
                flop = 12.0 if order == 2 else 18.0
                rec["fp64_frac"] = glups * flop / 1e3 / FP64_PEAK_TFLOPS
            probe[f"order{order}_{name}"] = rec
            sp.close()
            del sp
        del pp
    stage("forms: roofline_probe_16384")
    out["roofline_probe_16384"] = probe
    # time to 1e-6 relative error, 64^2 unit square, order 2, omega 10
    sq = G.unit_square_problem(64, 2, 10.0, seed=0)
    ref = WH.Solver(sq, stream=stream)
    ref.prepare()
    uref = torch.zeros(sq.n_total, dtype=torch.float64, device="cuda")
    ref.solve(uref, WH.GMRES, tol=1e-13, max_it=400, restart=200)
    solve = {}
    for name, prec, tol in (("fp64_gmres", WH.FP64, 1e-7), ("fp32_then_fp64_gmres", WH.FP32, 1e-7)):
        sv = WH.Solver(sq, stream=stream, precision=prec)
        sv.prepare()
        u = torch.zeros_like(uref)
        sv.solve(u, WH.GMRES, tol=tol, max_it=400, restart=200)  # warm-up (graphs)
        u.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = sv.solve(u, WH.GMRES, tol=tol, max_it=400, restart=200)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        err = float((u - uref).abs().max() / uref.abs().max())
        solve[name] = {"seconds": el, "rel_err_vs_reference": err, "wave_solves": st.iterations,
                       "residual": st.residual}
    solve["workload"] = ("64^2 unit square, order 2, omega 10, residual 1e-7; reference: FP64 "
                         "GMRES to 1e-13 (equal to the direct discrete solve in the tests)")
    stage("forms: solve_unit_square")
    out["solve_unit_square"] = solve
    stage("forms: deflation_disk512_omega20")
    out["deflation_disk512_omega20"] = measure_deflation(WH, G, torch, stream, periods=(1,),
                                                         tols=(1e-9, 1e-10))
    stage("forms: deflation on the 1024^2 omega 40 disk")
    # the headline workload solved to 1e-6 relative error: N_p = 4 (the paper runs 2-8),
    # 64 eigenpairs; plain GMRES does not converge there within the budget
    out["deflation_disk1024_omega40"] = measure_deflation(
        WH, G, torch, stream, nb=1024, nth=2048, nr=64, omega=40.0, k=64, periods=(4,),
        eig_budget=3000, plain_budget=600, extra_sources=2, tols=(1e-9, 1e-10))
    stage("forms: sphere-in-box")
    stage("forms: sphere_in_box_320")
    out["sphere_in_box_320"] = measure_sphere(WH, torch, stream, flush, cpu)
    stage("forms: 3D roofline probe")
    stage("forms: roofline_probe_3d_512")
    out["roofline_probe_3d_512"] = measure_cube_probe(WH, torch, stream)
    stage("forms: cube512_order4")
    out["cube512_order4"] = measure_cube_probe_o4(WH, torch, stream)
    return out


def _solve_timed(WH, torch, s, n, tol, max_it, restart=300):
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = s.solve(u, WH.GMRES, tol=tol, max_it=max_it, restart=restart)
    torch.cuda.synchronize()
    return u, {"seconds": time.perf_counter() - t0, "wave_solves": st.iterations,
               "wave_solves_fp32": st.products_fp32, "residual": st.residual,
               "converged": st.converged}


def measure_deflation(WH, G, torch, stream, nb=512, nth=1024, nr=32, omega=20.0, k=48,
                      periods=(1,), eig_budget=4000, plain_budget=3000, extra_sources=3,
                      tols=(1e-8,)):
    """Helmholtz solve time to 1e-6 relative error with deflation (Algorithm 3 through GMRES,
    Sec. 4.3-4.4) on the overset disk-in-square (nb^2 background + nth x nr annulus, order 4,
    c = 1), for N_p periods per iteration: k eigenpairs of S from the GPU eigensolver
    (wh_eigs, once per frequency), then deflated GMRES(300) to each residual tolerance in
    `tols` with the FP64 march and with FP32-then-FP64 wave solves, each checked against a
    deflated FP64 solve to 1e-12 (the reference); plain FP64 GMRES(300) with a fixed product
    budget for comparison; and `extra_sources` further seeded sources solved with the same
    eigenpairs (the paper's amortisation of the eigenpairs over several right-hand sides).
    The exact inflation's error is the basis's invariance residual ||S Q - Q T|| amplified by
    ||(I - T)^{-1}|| (about 1 / (1 - beta_max)), so both are measured (k more products) and
    reported with their product as the bound on the reference's error.  time_to_1e-6 is the
    eigensolve plus the first solve (loosest tolerance first) whose error against the
    reference is at most 1e-6, per precision."""
    import numpy as np
    prob = G.disk_problem(nb=nb, nth=nth, nr=nr, order=4, omega=omega, seed=0)
    n = prob.n_total
    out = {"workload": "disk-in-square %d^2 + %dx%d, order 4, omega %g, c = 1" % (nb, nth, nr, omega),
           "k": k}
    for Np in periods:
        rec = {}
        s = WH.Solver(prob, stream=stream, periods=Np)
        ti = s.prepare()
        rec["M"] = ti.M
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Q, T, beta, lam2, se = s.eigs(k, tol=1e-12, max_products=eig_budget, passes=1)
        torch.cuda.synchronize()
        rec["eigs"] = {"seconds": time.perf_counter() - t0, "wave_solves": se.iterations,
                       "converged": se.converged, "residual": se.residual,
                       "beta_max": float(np.max(beta)), "beta_k": float(np.min(np.abs(beta)))}
        SQ = torch.empty_like(Q)
        for i in range(k):
            s.iterate(Q[i].contiguous(), SQ[i], False)
        torch.cuda.synchronize()
        inv = float((SQ.T - Q.T @ torch.from_numpy(T).cuda()).abs().max())  # S q_j = sum_i T_ij q_i
        amp = float(np.linalg.norm(np.linalg.inv(np.eye(k) - T), 2))
        rec["eigs"].update({"invariance": inv, "inv_I_minus_T_norm": amp,
                            "inflation_error_bound": inv * amp})
        del SQ
        s.set_deflation_basis(Q, T)
        uref, rec["reference_1e-12"] = _solve_timed(WH, torch, s, n, 1e-12, 4000)
        nref = float(uref.abs().max())
        s32 = WH.Solver(prob, stream=stream, periods=Np, precision=WH.FP32)
        s32.prepare()
        s32.set_deflation_basis(Q, T)
        tts = {}
        for name, sv in (("fp64", s), ("fp32_then_fp64", s32)):
            for tol in tols:
                u, r = _solve_timed(WH, torch, sv, n, tol, 4000)
                r["rel_err"] = float((u - uref).abs().max()) / nref
                rec["deflated_%s_%g" % (name, tol)] = r
                if name not in tts and r["converged"] and r["rel_err"] <= 1e-6:
                    tts[name] = {"seconds": rec["eigs"]["seconds"] + r["seconds"], "tol": tol,
                                 "wave_solves": se.iterations + r["wave_solves"]}
                del u
        rec["time_to_1e-6"] = tts
        s32.close()
        s.set_deflation(None)
        up, rec["plain_fp64"] = _solve_timed(WH, torch, s, n, tols[0], plain_budget)
        rec["plain_fp64"]["rel_err"] = float((up - uref).abs().max()) / nref
        del up
        # more sources, same frequency: the eigenpairs are reused
        s.set_deflation_basis(Q, T)
        tot, prods = 0.0, 0
        for seed in range(1, extra_sources + 1):
            p2 = G.disk_problem(nb=nb, nth=nth, nr=nr, order=4, omega=omega, seed=seed)
            for gi in range(len(p2.grids)):
                s.set_forcing(gi, p2.f[gi])
            s.prepare()
            _, r = _solve_timed(WH, torch, s, n, tts.get("fp64", {}).get("tol", tols[-1]), 4000)
            tot += r["seconds"]
            prods += r["wave_solves"]
        rec["more_sources"] = {"sources": extra_sources, "seconds": tot, "wave_solves": prods}
        d = rec["deflated_fp64_%g" % tols[0]]
        rec["speedup_deflated_vs_plain_budget"] = rec["plain_fp64"]["seconds"] / d["seconds"]
        s.close()
        del Q, s, uref
        out["Np%d" % Np] = rec
    return out


def measure_cube_probe(WH, torch, stream):
    """The 3D half of the roofline probe: one Cartesian 512^3 grid on [0, 1]^3 (Dirichlet,
    omega 10, no interpolation, HBM resident), second order, FP64 and FP32: the march
    kernel's device time per launch over one iteration's steps; effective bandwidth counts
    the compulsory bytes of one update (49 B FP64, 33 B FP32: state, forcing, FP64 filter
    read and write, mask)."""
    from paper_2504_03074_gb300 import grids3 as G3
    hbm = float(measured_peaks().get("hbm_gbs", 6793.0))
    cube = G3.unit_cube_problem(512, omega=10.0)
    probe = {"workload": "unit cube 512^3, Dirichlet, omega 10, order 2, no interpolation",
             "hbm_peak_gbs": hbm}
    for name, prec, bpl in (("fp64", WH.FP64, 49.0), ("fp32", WH.FP32, 33.0)):
        sp = WH.Solver(cube, stream=stream, precision=prec)
        tp = sp.prepare()
        if prec == WH.FP32:
            sp.set_tuning(temporal_depth=1)  # the single-step march kernel on its own
        ms = sp.profile_kernels(reps=1)["march"][0]
        glups = tp.n_active / (ms * 1e-3) / 1e9
        rec = {"march_us": ms * 1e3, "value": glups, "unit": "GLUP/s", "M": tp.M,
               "effective_gbs": glups * bpl, "hbm_frac": glups * bpl / hbm}
        if prec == WH.FP64:
            rec["fp64_frac"] = glups * 15.0 / 1e3 / FP64_PEAK_TFLOPS
        probe[name] = rec
        if prec == WH.FP32:
            # temporal blocking: K steps per launch (the library's choice here), whole
            # iterations timed; path-level effective bandwidth = GLUP/s x 33 B (the k = 1
            # compulsory bytes); the blocked kernel's own algorithmic bytes per launch:
            # per point W^n, W^{n-1}, F (NaN-marked) 4 B each, V read + write 16 B, two
            # levels written 8 B = 36 B for K updates
            sp.set_tuning()
            t = sp.get_tuning()
            it = time_iterations(WH, torch, sp, cube.n_total, stream, None, 2)
            gl = tp.n_active * tp.M / it / 1e9
            pk = sp.profile_kernels(reps=1)
            bms, bn = pk["init"]  # [2] on three-dimensional contexts: the blocked march
            bbytes = t["blocked_points"] * 36.0
            probe["fp32_blocked"] = {
                "temporal_depth": t["temporal_depth"], "unit_depth": t["unit_depth"],
                "ms_per_iteration": it * 1e3, "value": gl, "unit": "GLUP/s",
                "path_effective_gbs": gl * 33.0, "path_hbm_frac": gl * 33.0 / hbm,
                "speedup_vs_single_step": gl / glups,
                "blocked_kernel_ms_per_launch": bms, "blocked_launches": bn,
                "blocked_kernel_gbs": bbytes / (bms * 1e-3) / 1e9,
                "blocked_kernel_hbm_frac": bbytes / (bms * 1e-3) / 1e9 / hbm,
                "blocked_bytes_per_update": 36.0 / t["temporal_depth"]}
        sp.close()
        del sp
    return probe


# Algorithmic FP64 FLOP per update of the three-dimensional order-4 march with the fused
# filter: 6 additions pairing symmetric neighbours, the centre multiply, 6 multiply-adds of
# the pair sums, the forcing multiply-add, the subtraction of W^{n-1}, the filter
# multiply-add = 6 + 1 + 12 + 2 + 1 + 2.
FLOP_PER_LUP_3D_O4 = 24.0


def measure_cube_probe_o4(WH, torch, stream):
    """Three-dimensional fourth order (Cartesian grids): one 512^3 grid on [0, 1]^3
    (Dirichlet, omega 10, two ghost layers, no interpolation, HBM resident), FP64 and FP32:
    the 13-point march kernel's device time per launch over one iteration's steps, and whole
    iterations (CUDA events, inputs larger than L2).  Effective bandwidth counts the
    compulsory bytes of one update as at second order (49 B FP64, 33 B FP32: state,
    forcing, FP64 filter read and write, mask); the four further neighbours per update
    come from cache."""
    from paper_2504_03074_gb300 import grids3 as G3
    hbm = float(measured_peaks().get("hbm_gbs", 6793.0))
    cube = G3.unit_cube_problem(512, omega=10.0, order=4)
    probe = {"workload": "unit cube 512^3, Dirichlet, omega 10, order 4, no interpolation",
             "hbm_peak_gbs": hbm}
    for name, prec, bpl in (("fp64", WH.FP64, 49.0), ("fp32", WH.FP32, 33.0)):
        sp = WH.Solver(cube, stream=stream, precision=prec)
        tp = sp.prepare()
        ms = sp.profile_kernels(reps=1)["march"][0]
        glups = tp.n_active / (ms * 1e-3) / 1e9
        it = time_iterations(WH, torch, sp, cube.n_total, stream, None, 2)
        rec = {"march_us": ms * 1e3, "value": glups, "unit": "GLUP/s", "M": tp.M,
               "effective_gbs": glups * bpl, "hbm_frac": glups * bpl / hbm,
               "ms_per_iteration": it * 1e3,
               "iteration_glups": tp.n_active * tp.M / it / 1e9}
        if prec == WH.FP64:
            rec["fp64_frac"] = glups * FLOP_PER_LUP_3D_O4 / 1e3 / FP64_PEAK_TFLOPS
        probe[name] = rec
        sp.close()
        del sp
    return probe


def measure_sphere(WH, torch, stream, flush, cpu=False):
    """The three-dimensional workload: sphere-in-box, 320^3 Cartesian background on
    [-2, 2]^3 + spherical shell 256 x 128 x 24 (polar band 15-165 degrees, width 0.3) + two
    orthographic pole patches 96^2 x 24, second order, Neumann sphere, Dirichlet box,
    omega 30, one seeded Gaussian source: one WaveHoltz iteration with the FP64 and with the
    FP32 march (GLUP/s, L2 flushed between iterations) and the device time per launch of
    the march and of the ghost-rule + interpolation kernel."""
    from paper_2504_03074_gb300 import grids3 as G3
    t0 = time.perf_counter()
    prob = G3.sphere_problem()
    res = {"workload": "sphere-in-box 320^3 + 256x128x24 + 2x96^2x24, order 2, omega 30",
           "points": prob.n_total, "active_points": prob.n_active,
           "receivers": prob.interp.n, "generate_s": time.perf_counter() - t0}
    for name, prec in (("fp64", WH.FP64), ("fp32", WH.FP32)):
        sp = WH.Solver(prob, stream=stream, precision=prec)
        tp = sp.prepare()
        t = time_iterations(WH, torch, sp, prob.n_total, stream, flush, 3)
        prof = sp.profile_kernels(reps=1)
        march_glups = tp.n_active / (prof["march"][0] * 1e-3) / 1e9
        rec = {"value": tp.n_active * tp.M / t / 1e9, "unit": "GLUP/s",
               "ms_per_iteration": t * 1e3, "M": tp.M,
               "march_ms_per_launch": prof["march"][0],
               "gather_ms_per_launch": prof["bc_gather"][0], "march_glups": march_glups}
        if prec == WH.FP64:  # 15 FP64 FLOP per 7-point update (stencil 10, forcing 3, filter 2)
            rec["march_fp64_frac"] = march_glups * 15.0 / 1e3 / FP64_PEAK_TFLOPS
        else:  # 33 compulsory bytes per update (W^n, W^{n-1} r/w, F, V r/w, mask)
            hbm = float(measured_peaks().get("hbm_gbs", 6793.0))
            rec["march_hbm_frac"] = march_glups * 33.0 / hbm
            rec["layout"] = sp.get_tuning()
            # the autotuner over temporal depth 1..4 and unit depths (blocked march)
            tune = sp.autotune(reps=1)
            ta = time_iterations(WH, torch, sp, prob.n_total, stream, flush, 3)
            pk = sp.profile_kernels(reps=1)
            rec["autotuned"] = {
                "temporal_depth": tune["temporal_depth"], "unit_depth": tune["unit_depth"],
                "blocked_points": tune["blocked_points"], "candidates": tune["candidates"],
                "value": tp.n_active * tp.M / ta / 1e9, "ms_per_iteration": ta * 1e3,
                "path_hbm_frac": tp.n_active * tp.M / ta / 1e9 * 33.0 / hbm,
                "single_step_march_ms": pk["march"], "gather_ms": pk["bc_gather"],
                "blocked_march_ms": pk["init"]}
        res[name] = rec
        sp.close()
        del sp
    res["speedup_fp32_vs_fp64"] = res["fp32"]["value"] / res["fp64"]["value"]
    # time to a 1e-3 relative GMRES residual from zero (GMRES(150)); 1e-6 needs more than
    # 3,000 wave solves here at N_p = 1 (measured once: residual 1.2e-5 after 3,000)
    solve = {"tol": 1e-3, "restart": 150}
    for name, prec in (("fp32_then_fp64", WH.FP32), ("fp64", WH.FP64)):
        sp = WH.Solver(prob, stream=stream, precision=prec)
        sp.prepare()
        u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = sp.solve(u, WH.GMRES, tol=1e-3, max_it=600, restart=150)
        torch.cuda.synchronize()
        solve[name] = {"seconds": time.perf_counter() - t0, "converged": st.converged,
                       "residual": st.residual, "wave_solves_fp32": st.products_fp32,
                       "wave_solves_fp64": st.products_fp64}
        sp.close()
        del sp, u
    solve["speedup_fp32_vs_fp64"] = solve["fp64"]["seconds"] / solve["fp32_then_fp64"]["seconds"]
    res["solve_to_1e-3"] = solve
    if cpu:  # the 3D oracle on the half-resolution sample of the same recipe: one thread,
        # then all cores (the same source built with OpenMP; equal results checked)
        import numpy as np
        from oracle import oracle3 as O3
        half = G3.sphere_problem(nb=160, nphi=128, nth=64, nr=12, npatch=48)
        orc = O3.Oracle3(half)
        v = G3.random_state3(half, 1)
        t0 = time.perf_counter()
        ref = orc.iterate(v, True)
        el = time.perf_counter() - t0
        lups = half.n_active * orc.time.M
        rec = {"value": lups / el / 1e9, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "seconds": el, "host": host_cpu(),
               "single_thread": {"value": lups / el / 1e9, "seconds": el, "cores": 1},
               "sample": "one oracle WaveHoltz iteration of the half-resolution sample "
                         "(160^3 + 128x64x12 + 2x48^2x12, M=%d)" % orc.time.M}
        try:
            omp = O3.Oracle3(half, openmp=True)
            t0 = time.perf_counter()
            out = omp.iterate(v, True)
            eln = time.perf_counter() - t0
            threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
            rec.update({"value": lups / eln / 1e9, "cores": threads, "seconds": eln,
                        "all_cores": {"value": lups / eln / 1e9, "seconds": eln,
                                      "cores": threads,
                                      "equals_single_thread": bool(np.array_equal(out, ref))}})
        except Exception as e:
            rec["all_cores"] = {"unavailable": str(e)[:200]}
        res["cpu_baseline"] = rec
    return res


def run_reference(args):
    """--impl reference: the CPU oracle on the host cores, same metric/unit/config; each
    step is one oracle WaveHoltz iteration on the half-resolution sample of the workload
    (512^2 + 1024x32, same recipe, omega = 40), so the whole run stays within minutes."""
    r, w, _ = rank_info()
    if r != 0:
        return 0
    from oracle import oracle as O
    from paper_2504_03074_gb300 import grids as G
    prob = G.disk_problem(nb=512, nth=1024, nr=32, order=4, omega=40.0, seed=0)
    orc = O.Oracle(prob)
    v = orc.zeros()
    for _ in range(args.warmup):
        v = orc.iterate(v, True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v = orc.iterate(v, True)
    el = time.perf_counter() - t0
    lups = prob.n_active * orc.time.M * args.steps
    val = lups / el / 1e9
    sample = ("one oracle WaveHoltz iteration per step on the half-resolution sample "
              "(512^2 + 1024x32 annulus, order 4, omega 40, M=%d steps)" % orc.time.M)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GLUP/s",
        "n_gpus": w, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": val,
                         "unit": "GLUP/s", "host": host_cpu()},
        "e2e": {"value": val, "unit": "GLUP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))
    return 0


def run_profile_case(case):
    """A fixed small workload for ncu captures (no timing, no JSON line)."""
    import torch
    from paper_2504_03074_gb300 import build as B
    B.build()
    from paper_2504_03074_gb300 import grids as G, waveholtz as WH
    prec = WH.FP32 if case.startswith("fp32") else WH.FP64
    if case.endswith("sphere320"):
        from paper_2504_03074_gb300 import grids3 as G3
        sp = G3.sphere_problem()
        s = WH.Solver(sp, precision=prec)
        ti = s.prepare()
        a = torch.zeros(sp.n_total, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        s.iterate(a, b, True)
        torch.cuda.synchronize()
        print(f"profile case {case}: {sp.n_total} points, 1 iteration ({ti.M} march launches)")
        return 0
    if case.startswith("fp32_cube320"):
        from paper_2504_03074_gb300 import grids3 as G3
        cp = G3.unit_cube_problem(320, omega=10.0)
        s = WH.Solver(cp, precision=prec)
        ti = s.prepare()
        if case.endswith("single"):
            s.set_tuning(temporal_depth=1)
        a = torch.zeros(cp.n_total, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        s.iterate(a, b, True)
        torch.cuda.synchronize()
        print(f"profile case {case}: {cp.n_total} points, 1 iteration, layout {s.get_tuning()}")
        return 0
    if case.endswith("square8192"):
        sq = G.unit_square_problem(8192, 4, 10.0, seed=0)
        s = WH.Solver(sq, precision=prec)
        s.prepare()
        s.profile_kernels(reps=5)  # march launches only (the first step of an iteration)
        torch.cuda.synchronize()
        print(f"profile case {case}: {sq.n_total} points, 5 march launches")
        return 0
    bp, _ = G.batch_disk_problem(16, seed=100)
    s = WH.Solver(bp, precision=prec)
    s.prepare()
    a = torch.zeros(bp.n_total, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    for _ in range(3):
        s.iterate(a, b, True)
        a, b = b, a
    torch.cuda.synchronize()
    print(f"profile case {case}: {bp.n_total} points, 3 iterations")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--small", action="store_true", help="small workload (profiling)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP32 / batched / solve-time measurements")
    ap.add_argument("--profile-case",
                    choices=["fp32_batch16", "fp64_batch16", "fp32_square8192",
                             "fp64_square8192", "fp32_sphere320", "fp64_sphere320",
                             "fp32_cube320_blocked", "fp32_cube320_single"],
                    help="profiling aid: a 16-instance disk-in-square batch (8.4 M points, "
                         "3 iterations), one 8192^2 order-4 Cartesian grid (67 M points, "
                         "5 march launches), the 3D sphere-in-box (34 M points, one "
                         "iteration) or a 320^3 cube with the blocked or the single-step "
                         "FP32 march, HBM resident, in one precision; no bench line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args.profile_case)

    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = rank_info()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2504_03074_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2504_03074_gb300 import grids as G
    from paper_2504_03074_gb300 import waveholtz as WH

    if args.small:
        prob = G.disk_problem(nb=256, nth=512, nr=16, order=4, omega=20.0, seed=rank)
    else:
        prob = G.disk_problem(nb=1024, nth=2048, nr=64, order=4, omega=40.0, seed=rank)
    stream = torch.cuda.Stream()
    s = WH.Solver(prob, stream=stream)
    ti = s.prepare()
    n = prob.n_total
    lups = ti.n_active * ti.M
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    va = torch.zeros(n, dtype=torch.float64, device="cuda")
    vb = torch.empty_like(va)
    with torch.cuda.stream(stream), ClockSampler(local) as clk:
        clk.wait_first()
        for _ in range(max(args.warmup, 0)):
            s.iterate(va, vb, True)
            va, vb = vb, va
        stream.synchronize()
        if world > 1:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        torch.cuda.synchronize()
        clk_start = clk.mark()
        for k in range(args.steps):
            flush.fill_(float(k))  # L2 flush between timed iterations (untimed)
            ev[k][0].record(stream)
            s.iterate(va, vb, True)
            ev[k][1].record(stream)
            va, vb = vb, va
        stream.synchronize()
        torch.cuda.synchronize()
        launches = s.last_launch_count() * args.steps
    ms = [a.elapsed_time(b) for a, b in ev]
    t_local = sum(ms) / 1e3
    value, t_max = whole_job(lups * args.steps, t_local, world)

    # end-to-end through the public API with host buffers (pinned), copies inside
    hin = torch.zeros(n, dtype=torch.float64).pin_memory()
    hout = torch.empty(n, dtype=torch.float64).pin_memory()
    hin.copy_(va.cpu())
    e2e_ms = []
    for k in range(max(3, min(args.steps, 5))):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.iterate_host_buffers(hin, hout, True)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        hin, hout = hout, hin
    e2e_t = statistics.median(e2e_ms) / 1e3
    e2e_val = lups * world / e2e_t / 1e9

    # per-kernel device times: graph-captured bursts of back-to-back launches, events on
    # the library's stream
    prof = s.profile_kernels(50)
    march_ms, march_n = prof["march"]
    avg_march_s = march_ms / 1e3
    flops_per_launch = FLOP_PER_LUP_O4 * ti.n_active  # every launch updates all points
    achieved = flops_per_launch / avg_march_s / 1e12
    total_prof = sum(v[0] * v[1] for v in prof.values())
    # the FP64 roofline measured here, on this GPU, right after the timed region: a kernel
    # of independent FMA chains and nothing else (wh_probe_fp64), best of 5 launches, with
    # the clocks sampled during it
    global FP64_PEAK_TFLOPS
    stage("FP64 probe")
    with ClockSampler(local) as pclk:
        pclk.wait_first()
        pmark = pclk.mark()
        peak_tf, peak_ms = WH.probe_fp64(5)
    FP64_PEAK_TFLOPS = peak_tf
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tf,
                "unit": "TFLOP/s", "frac": achieved / peak_tf,
                "traffic": recorded_traffic("march_kernel"),
                "kernel": "march_kernel<double,4>", "avg_launch_us": avg_march_s * 1e6,
                "flop_per_launch": flops_per_launch,
                "share_of_iteration": march_ms * march_n / total_prof,
                "peak_source": "measured in this run: wh_probe_fp64 (independent DFMA chains, "
                               "FMA = 2 FLOP, best of 5 launches of %.2f ms)" % peak_ms,
                "peak_clocks": pclk.summary(pmark),
                "nominal_fp64_tflops": 1.25}

    stage("main line done")
    forms = None
    if not args.no_forms and not args.small and rank == 0:  # only rank 0 prints them
        forms = measure_forms(WH, G, torch, prob, stream, flush, rank,
                              cpu=world == 1 and not args.no_cpu_baseline)

    stage("forms done")
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.small:
        stage("cpu baseline")
        cpu = cpu_baseline(prob, "one full oracle WaveHoltz iteration (M=%d steps) of the "
                                 "same workload, single thread and all host cores" % ti.M)
    out = {
        "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if not args.small else "small 256^2+512x16 o4",
                   "M": ti.M, "Nt": ti.Nt, "dt": ti.dt, "n_active": ti.n_active,
                   "n_total": ti.n_total, "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "GLUP/s", "h2d_bytes_per_step": n * 8,
                "d2h_bytes_per_step": n * 8, "ms_per_step": e2e_t * 1e3},
        "clocks": clk.summary(clk_start),
        "gpu_launches": launches,
        "forms": forms,
        "kernels_ms_per_iteration": {k: v[0] * v[1] for k, v in prof.items()},
        "kernels_us_per_launch": {k: v[0] * 1e3 for k, v in prof.items()},
    }
    if rank == 0:
        print(json.dumps(out))
    s.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
