"""Throughput of the adaptive multigrid Wilson-Dirac solve on GB300.

Workload (three-level sweep point, 2d U(1) Schwinger model): 256 x 256 periodic
lattice, quenched links from 2000 Metropolis sweeps (cold start, 10 hits,
step 0.5 rad) at beta in {3, 6, 10}; for each beta the adaptive setup (4x4 then
2x2 blocks, Nv = 8, 5 passes, MR 4 + 4, omega 0.8) runs once at the lightest
mass m_c + 0.005 and is reused for m_c + 0.02 and m_c + 0.1; one Gaussian source
per mass, solved to a 1e-10 true residual by FP64 flexible GCR.

One step = the three setups and nine solves (the whole hot path once over the
batch). The metric is MG solves per second including setup. The default run
uses the mixed-precision V-cycle (FP32 inside the FP64 outer loop); the all-FP64
solver is timed beside it. L2 is flushed (512 MiB write) before every timed step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs the same per-rank workload with its own seeds
(independent solves: weak scaling, no data-path collective); rank 0 prints one
JSON line with the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402

L = 256
BETAS = (3.0, 6.0, 10.0)
DMS = (0.005, 0.02, 0.1)
TOL = 1e-10
WORKLOAD_ID = 1
METRIC = "MG solves/s to 1e-10 true residual (incl. setup)"
WORKLOAD = ("2d U(1) Wilson-Dirac 256x256, beta in {3,6,10}, m-m_c in {0.005,0.02,0.1}; "
            "3-level MG 4x4/2x2 Nv=8, 5 passes, MR 4+4; setup once per beta, 9 solves per step")


# outer GCR restart of the sweep: 8 at 256^2 (a step took 90.5 ms against 93.0 ms with 16: the FP64
# Gram-Schmidt over the basis is a tenth of an outer iteration, for 0 to 6 more outer iterations per
# solve); the 1024^2 points keep 16 (with 8 the beta 6 field at m_c + 0.005 did not converge in 3000)
OUTER_RESTART = {256: 8, 1024: 16}


def mg_params(precision: int, L_field: int = 256):
    import paper_0707_4018_gb300 as mg
    # max_iter 3000: the 1024^2 field at m_c(256^2) + 0.005 needs about 500 outer iterations
    return mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=precision,
                                coarsest_tol=0.2, coarsest_restart=16, max_iter=3000,
                                gcr_restart=OUTER_RESTART.get(L_field, 16))


def mcrit_table():
    return json.load(open(os.path.join(ROOT, "tests", "golden", "mcrit.json")))


def make_inputs(rank: int, Lf: int = L):
    """Links, critical masses and sources of the workload (host numpy). The links come from the
    GPU twin of the Metropolis generator (the CPU chain, step for step); the digest of every
    field is compared with the one the CPU generator stored next to its critical mass."""
    table = mcrit_table()
    fields = []
    wid = WORKLOAD_ID + 100 * rank
    for beta in BETAS:
        (U, theta, _), = inputs.schwinger_links_gpu(Lf, beta, sweeps=2000, workload_id=wid)
        row = table.get(f"w{WORKLOAD_ID}_L{Lf}_b{beta:g}")
        if row is None:
            raise RuntimeError(f"no critical mass stored for L={Lf} beta={beta}")
        digest_ok = rank == 0 and row["theta_digest"] == inputs.field_digest(theta)
        seed = inputs.workload_seed(wid, Lf, beta)
        chis = [inputs.gaussian_source(Lf, Lf, seed=seed, index=i) for i in range(len(DMS))]
        fields.append(dict(beta=beta, L=Lf, U=U, m_c=row["m_crit"], m_c_from=row.get("m_crit_from"),
                           digest_ok=digest_ok, chis=chis))
    return fields


def device_fields(fields):
    import torch
    out = []
    for f in fields:
        Lf = f["L"]
        out.append(dict(beta=f["beta"], L=Lf, m_c=f["m_c"], U_dev=torch.from_numpy(f["U"]).cuda(),
                        chi_dev=[torch.from_numpy(c).cuda() for c in f["chis"]],
                        psi_dev=[torch.empty((Lf * Lf, 2), dtype=torch.complex128, device="cuda") for _ in DMS],
                        U_host=torch.from_numpy(f["U"]).pin_memory(),
                        chi_host=[torch.from_numpy(c).pin_memory() for c in f["chis"]]))
    return out


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _one_field(f, precision, stats_out, host_io, contexts):
    """One beta: setup at the lightest mass and the three solves. Concurrent mode: the setup is
    cloned for the two heavier masses (mg_clone rebuilds the Galerkin operators) and the three
    solves run at once, one host thread and context stream each; serial mode: update_mass
    between the solves."""
    import paper_0707_4018_gb300 as mg
    if host_io is not None:
        U = f["U_host"].to("cuda", non_blocking=True)
    else:
        U = f["U_dev"]
    Lf = f.get("L", L)
    ctx = mg.Context.setup(U, f["m_c"] + DMS[0], (Lf, Lf), mg_params(precision, Lf))
    contexts.append(ctx)

    def solve(c, i, dm):
        chi = f["chi_host"][i].to("cuda", non_blocking=True) if host_io is not None else f["chi_dev"][i]
        psi = f["psi_dev"][i]
        st = c.solve(chi, psi, TOL)
        if host_io is not None:
            host_io[f["beta"]][i].copy_(psi, non_blocking=True)
        if stats_out is not None:
            stats_out.append(dict(beta=f["beta"], dm=dm, **st))

    if not CONCURRENT:
        for i, dm in enumerate(DMS):
            if i > 0:
                ctx.update_mass(f["m_c"] + dm)
            solve(ctx, i, dm)
        return len(DMS)
    ctxs = [ctx] + [ctx.clone(f["m_c"] + dm) for dm in DMS[1:]]
    contexts.extend(ctxs[1:])
    errors = []

    def work(i):
        try:
            solve(ctxs[i], i, DMS[i])
        except BaseException as e:  # re-raised on the calling thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(DMS))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return len(DMS)


# The betas (and, through clones of a beta's setup, its masses) are independent problems with
# their own contexts (own streams): one host thread each lets their small, latency-bound
# kernels overlap on the GPU. --serial runs them in turn.
CONCURRENT = True


def run_step_graph(fields_dev, precision: int, stats_out=None, host_io=None):
    """One pass over the batch with device-driven outer loops: one host thread per beta runs the
    beta's setup, the clones of it for the heavier masses, then one mg_solve_multi launch for the
    beta's three solves (each outer loop a conditional WHILE node on the device). The betas run
    concurrently, so one beta's setup overlaps another's solves on the GPU."""
    import torch
    import paper_0707_4018_gb300 as mg
    results, errors = {}, []

    def run(f):
        cs = []
        try:
            U = f["U_host"].to("cuda", non_blocking=True) if host_io is not None else f["U_dev"]
            Lf = f.get("L", L)
            c = mg.Context.setup(U, f["m_c"] + DMS[0], (Lf, Lf), mg_params(precision, Lf))
            cs = [c] + [c.clone(f["m_c"] + dm) for dm in DMS[1:]]
            chis = [f["chi_host"][i].to("cuda", non_blocking=True) if host_io is not None else f["chi_dev"][i]
                    for i in range(len(DMS))]
            st = mg.solve_multi(cs, chis, f["psi_dev"], TOL)
            if host_io is not None:
                for i, psi in enumerate(f["psi_dev"]):
                    host_io[f["beta"]][i].copy_(psi, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            results[f["beta"]] = st
        except BaseException as e:  # re-raised on the calling thread
            errors.append(e)
        finally:
            for c in cs:
                c.close()

    threads = [threading.Thread(target=run, args=(f,)) for f in fields_dev]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    if stats_out is not None:
        for f in fields_dev:
            stats_out.extend(dict(beta=f["beta"], dm=dm, **s) for dm, s in zip(DMS, results[f["beta"]]))
    return sum(len(v) for v in results.values())


# how a step runs its solves: "graph" (one mg_solve_multi launch for all of them) or "threads"
# (one host thread and host-driven loop per solve)
STEP_MODE = "graph"


def run_step(fields_dev, precision: int, stats_out=None, host_io=None):
    """One pass over the batch: per beta, setup at the lightest mass and three solves."""
    import torch
    if STEP_MODE == "graph" and CONCURRENT:
        return run_step_graph(fields_dev, precision, stats_out, host_io)
    contexts = []
    stats = [] if stats_out is not None else None
    if CONCURRENT and len(fields_dev) > 1:
        errors, counts = [], []

        def work(f):
            try:
                counts.append(_one_field(f, precision, stats, host_io, contexts))
            except BaseException as e:  # re-raised on the calling thread
                errors.append(e)

        threads = [threading.Thread(target=work, args=(f,)) for f in fields_dev]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        n_solves = sum(counts)
    else:
        n_solves = sum(_one_field(f, precision, stats, host_io, contexts) for f in fields_dev)
    torch.cuda.current_stream().synchronize()
    for ctx in contexts:  # freed after every beta finished (a free synchronises the device)
        ctx.close()
    if stats_out is not None:
        stats_out.extend(sorted(stats, key=lambda d: (d["beta"], d["dm"])))
    return n_solves


def timed_steps(fields_dev, precision, steps, warmup, flush, dist_ctx, host_io=None, sampler=None):
    import torch
    import paper_0707_4018_gb300 as mg
    for _ in range(warmup):
        run_step(fields_dev, precision, host_io=host_io)
    stats = []
    barrier(dist_ctx)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    launches0 = mg.mg_kernel_launches()
    total_ms = 0.0
    solves = 0
    stream = torch.cuda.current_stream()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solves += run_step(fields_dev, precision, stats_out=stats, host_io=host_io)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    launches = mg.mg_kernel_launches() - launches0
    clocks = sampler.stop() if sampler else None
    barrier(dist_ctx)
    total_ms = max_over_ranks(total_ms, dist_ctx)
    return dict(ms=total_ms, solves=solves, stats=stats, launches=launches, clocks=clocks)


LARGE_L = 1024


PREC_NAMES = {0: "fp64", 1: "mixed", 2: "fp16"}


def config1_large(flush, precisions=(1, 2, 0)):
    """The 1024^2 points of the three-level sweep (beta in {3, 6, 10}, m - m_c in {0.005, 0.02,
    0.1}): one step (3 setups + 9 solves, betas and masses concurrently as in the headline) after
    one untimed step, per precision. m_c is the 256^2 calibration of the same beta (the 1024^2
    spectrum is beyond the oracle's Arnoldi scan)."""
    import torch
    fields = make_inputs(0, LARGE_L)
    fdev = device_fields(fields)
    out = {"lattice": f"{LARGE_L}x{LARGE_L}", "m_c_from": [f["m_c_from"] for f in fields],
           "gauge_digest_matches_table": all(f["digest_ok"] for f in fields)}
    stream = torch.cuda.current_stream()
    sols = {}
    for prec in precisions:
        run_step(fdev, prec)
        flush.zero_()
        stats = []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n = run_step(fdev, prec, stats_out=stats)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        sols[prec] = [[p.clone() for p in f["psi_dev"]] for f in fdev]
        out[PREC_NAMES[prec]] = dict(
            value=n / (ms * 1e-3), unit="solves/s (incl. setup)", ms_per_step=ms, solves=n,
            iters=[s["iters"] for s in stats], converged=all(s["converged"] for s in stats),
            worst_true_rel_residual=max(s["true_rel_residual"] for s in stats),
            setup_s=sorted({round(s["setup_s"], 4) for s in stats}))
    if 0 in sols and 1 in sols:
        out["mixed_vs_fp64_rel_diff"] = solution_diffs(sols[1], sols[0])
    if 0 in sols and 2 in sols:
        out["fp16_vs_fp64_rel_diff"] = solution_diffs(sols[2], sols[0])
    return out


def solution_diffs(a, b):
    """|psi_a - psi_b| / |psi_b| per (beta, mass) of a step: the mixed-precision result against the
    all-FP64 one (both solved to the 1e-10 true residual)."""
    import torch
    return [[float(torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(y)) for x, y in zip(fa, fb)]
            for fa, fb in zip(a, b)]


LEARN_L, LEARN_TRAIN, LEARN_EVAL, LEARN_BIG_L, LEARN_BIG_EVAL = 128, 256, 64, 512, 8
LEARN_WID = 4


def learned_setup_eval(n_train: int = LEARN_TRAIN, n_eval: int = LEARN_EVAL, n_big: int = LEARN_BIG_EVAL,
                       steps: int = 300, nu_refine: int = 16, max_rate: float = 0.6):
    """Learned near-null setup (2 levels, 4x4 blocks, Nv 8, beta 6): the network is trained on the
    plain adaptive setup's prolongators of n_train fields at 128^2, then held-out fields at 128^2
    and 512^2 are set up both ways (plain: 5 passes; learned: the network's vectors, nu_refine MR
    iterations, the convergence-rate judge with the plain setup as fallback) and solved once each
    to 1e-10 at m = m_c + 0.02 (m_c: the stored 128^2 field, and the 256^2 calibration for 512^2)."""
    import torch
    import paper_0707_4018_gb300 as mg
    table = mcrit_table()
    t0 = time.time()
    seeds = [inputs.member_seed(LEARN_WID, LEARN_L, 6.0, i) for i in range(n_train + n_eval)]
    th, _ = inputs.metropolis_u1_2d_gpu(LEARN_L, LEARN_L, [6.0] * len(seeds), seeds, 2000)
    big_seeds = [inputs.member_seed(LEARN_WID, LEARN_BIG_L, 6.0, i) for i in range(n_big)]
    thb, _ = inputs.metropolis_u1_2d_gpu(LEARN_BIG_L, LEARN_BIG_L, [6.0] * n_big, big_seeds, 2000)
    gen_s = time.time() - t0
    U = torch.from_numpy(np.stack([inputs.links_from_angles(t) for t in th])).cuda()
    Ub = torch.from_numpy(np.stack([inputs.links_from_angles(t) for t in thb])).cuda()
    m = table["w2_L128_b6"]["m_crit"] + 0.02
    mb = table["w1_L256_b6"]["m_crit"] + 0.02
    plain_p = mg.mg_default_params(levels=2, blocks=[(4, 4)], Nv=[8], n_pass=5, precision=1, coarsest_tol=0.2)
    learn_p = mg.mg_default_params(levels=2, blocks=[(4, 4)], Nv=[8], n_pass=1, precision=1, coarsest_tol=0.2)
    torch.cuda.synchronize()
    t0 = time.time()
    targets = []
    for i0 in range(0, n_train, 64):
        cs = mg.Context.setup_batch([U[i] for i in range(i0, min(n_train, i0 + 64))], [m] * min(64, n_train - i0),
                                    [(LEARN_L, LEARN_L)] * min(64, n_train - i0), [plain_p] * min(64, n_train - i0))
        targets += [c.prolongator(0) for c in cs]
        for c in cs:
            c.close()
    T = torch.stack(targets)
    torch.cuda.synchronize()
    target_s = time.time() - t0
    net = mg.NullNet(8, 16, 8, seed=ROOT_NET_SEED)
    t0 = time.time()
    losses = net.train(U[:n_train], (LEARN_L, LEARN_L), T, (4, 4), steps=steps, batch=16, lr=3e-3, seed=5)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    del T

    def compare(Us, Lf, mass, count, tag):
        chi = torch.from_numpy(inputs.gaussian_source(Lf, Lf, seed=11)).cuda()
        psi = torch.empty_like(chi)
        rows = {"plain": [], "learned": [], "plain_fp64": []}
        fallbacks = 0
        for i in range(count):
            for kind in ("plain", "learned", "plain_fp64"):
                torch.cuda.synchronize()
                t = time.time()
                if kind == "learned":
                    ctx, used, rate = mg.Context.setup_learned(Us[i], mass, (Lf, Lf), learn_p, net,
                                                               noise_seed=1000 + i, nu_refine=nu_refine,
                                                               max_rate=max_rate)
                    fallbacks += 0 if used else 1
                else:
                    q = plain_p if kind == "plain" else mg.mg_default_params(levels=2, blocks=[(4, 4)], Nv=[8],
                                                                             n_pass=5, precision=0,
                                                                             coarsest_tol=0.2)
                    ctx = mg.Context.setup(Us[i], mass, (Lf, Lf), q)
                st = ctx.solve(chi, psi, TOL)
                torch.cuda.synchronize()
                rows[kind].append(dict(iters=st["iters"], setup_s=st["setup_s"], solve_s=st["solve_s"],
                                       wall_s=time.time() - t, res=st["true_rel_residual"],
                                       conv=st["converged"]))
                ctx.close()
        out = {"lattice": f"{Lf}x{Lf}", "held_out_fields": count, "learned_fallbacks": fallbacks}
        for kind, r in rows.items():
            out[kind] = dict(mean_iters=float(np.mean([x["iters"] for x in r])),
                             mean_setup_ms=1e3 * float(np.mean([x["setup_s"] for x in r])),
                             mean_solve_ms=1e3 * float(np.mean([x["solve_s"] for x in r])),
                             solves_per_s_incl_setup=len(r) / sum(x["wall_s"] for x in r),
                             all_converged=all(x["conv"] for x in r),
                             worst_true_rel_residual=max(x["res"] for x in r))
        return out

    small = compare([U[n_train + i] for i in range(n_eval)], LEARN_L, m, n_eval, "128")
    big = compare([Ub[i] for i in range(n_big)], LEARN_BIG_L, mb, n_big, "512")
    return {"train": {"fields": n_train, "lattice": f"{LEARN_L}x{LEARN_L}", "steps": steps, "batch": 16,
                      "loss_first10": float(np.mean(losses[:10])), "loss_last10": float(np.mean(losses[-10:])),
                      "gen_s": gen_s, "plain_setups_s": target_s, "train_s": train_s},
            "learned": {"nu_refine": nu_refine, "n_pass": 1, "judge_max_rate": max_rate},
            "eval_128": small, "eval_512": big,
            "mass": "m_c + 0.02 (m_c of the stored 128^2 beta 6 field; 256^2 calibration for 512^2)"}


ROOT_NET_SEED = 20070704

C2_FIELDS, C2_RHS, C2_SIZES, C2_WID = 32, 16, (128, 256, 512, 1024), 2
C2_WAVE_SITES = 4 * 1024 * 1024  # sites set up and solved together (device memory of the batched bases)


def config2_sizes(n_fields: int = C2_FIELDS):
    """Lattice sizes of the many-configuration batch: uniform draws from {128, 256, 512, 1024}
    (the inputs module's counter-based uniforms, key root seed + 2)."""
    u = inputs.uniform(n_fields, inputs.ROOT_SEED + C2_WID, 0xC2)
    return [C2_SIZES[min(3, int(x * 4))] for x in u]


def config2_batch(n_fields: int = C2_FIELDS, nrhs: int = C2_RHS, precision: int = 1):
    """Many configurations x many right-hand sides: n_fields beta 6 fields with sizes from
    config2_sizes, nrhs Gaussian sources each, m = m_c + 0.02 (m_c of the stored 128^2 field for
    128^2 and the 256^2 calibration above). Fields are processed in waves of at most 4 M sites: the
    wave's setups run at once (mg_setup_batch), then every solve of the wave (fields x sources) runs
    from one graph launch (mg_solve_multi; each context's nrhs vectors in lockstep inside its WHILE
    loop, the coarse residual applies on tensor cores). Timed end to end including setup."""
    import torch
    import paper_0707_4018_gb300 as mg
    table = mcrit_table()
    sizes = config2_sizes(n_fields)
    mc = {128: table["w2_L128_b6"]["m_crit"]}
    for Lf in C2_SIZES[1:]:
        mc[Lf] = table["w1_L256_b6"]["m_crit"]
    fields = []
    t0 = time.time()
    for Lf in sorted(set(sizes)):
        idx = [i for i, s in enumerate(sizes) if s == Lf]
        seeds = [inputs.member_seed(C2_WID, Lf, 6.0, i) for i in idx]
        th, _ = inputs.metropolis_u1_2d_gpu(Lf, Lf, [6.0] * len(idx), seeds, 2000)
        for k, i in enumerate(idx):
            U = torch.from_numpy(inputs.links_from_angles(th[k])).cuda()
            chi = torch.stack([torch.from_numpy(inputs.gaussian_source(Lf, Lf, seed=seeds[k], index=v))
                               for v in range(nrhs)]).cuda()
            fields.append(dict(i=i, L=Lf, U=U, chi=chi, psi=torch.empty_like(chi)))
    gen_s = time.time() - t0
    fields.sort(key=lambda f: -f["L"])
    waves, cur, sites = [], [], 0
    for f in fields:
        if cur and sites + f["L"] ** 2 > C2_WAVE_SITES:
            waves.append(cur)
            cur, sites = [], 0
        cur.append(f)
        sites += f["L"] ** 2
    waves.append(cur)
    p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=precision, coarsest_tol=0.2,
                             max_rhs=nrhs, gcr_restart=8)
    stats = []
    serial_setups = 0
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for wave in waves:
        try:
            ctxs = mg.Context.setup_batch([f["U"] for f in wave], [mc[f["L"]] + 0.02 for f in wave],
                                          [(f["L"], f["L"]) for f in wave], [p] * len(wave))
        except mg.MGError as e:  # a bounded device wait ran out under contention: set up one by one
            if e.code != 8:
                raise
            serial_setups += 1
            ctxs = [mg.Context.setup(f["U"], mc[f["L"]] + 0.02, (f["L"], f["L"]), p) for f in wave]
        st = mg.solve_multi(ctxs, [f["chi"] for f in wave], [f["psi"] for f in wave], TOL,
                            nrhs=[nrhs] * len(wave), raise_on_fail=False)
        stats += st
        for c in ctxs:
            c.close()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    n_solves = n_fields * nrhs
    return {"fields": n_fields, "sources_per_field": nrhs, "sizes": {str(Lf): sizes.count(Lf) for Lf in C2_SIZES},
            "waves": len(waves), "waves_set_up_one_by_one": serial_setups, "solves": n_solves,
            "value": n_solves / (ms * 1e-3),
            "unit": "solves/s (incl. setup)", "ms": ms, "gen_s": gen_s,
            "all_converged": all(s["converged"] for s in stats),
            "worst_true_rel_residual": max(s["true_rel_residual"] for s in stats),
            "mean_iters": float(np.mean([s["iters"] for s in stats])),
            "precision": "FP64 outer GCR (device-driven, gcr_restart 8), FP32 cycles, coarse residual applies "
                         "on tensor cores (BF16 operands, FP32 sums)"}


def dslash_roofline(precision: int, L_big: int = 4096, iters: int = 20):
    """Fine Wilson apply alone on a lattice far larger than L2: algorithmic bytes / time."""
    import torch
    import paper_0707_4018_gb300 as mg
    dt = torch.complex128 if precision == 0 else torch.complex64
    V = L_big * L_big
    g = torch.Generator(device="cuda").manual_seed(5)
    ang = torch.rand((V, 2), device="cuda", generator=g, dtype=torch.float64) * 2 * np.pi
    U = torch.polar(torch.ones_like(ang), ang).to(dt)
    psi = torch.randn((V, 2), device="cuda", generator=g, dtype=dt)
    out = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        mg.mg_dslash(U, psi, out, 0.01, (L_big, L_big), precision)
    ms = []
    for _ in range(iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mg.mg_dslash(U, psi, out, 0.01, (L_big, L_big), precision)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms) * 1e-3
    cplx = 16 if precision == 0 else 8
    bytes_alg = V * 6 * cplx  # psi in (2), U (2), psi out (2) complex per site
    return dict(lattice=f"{L_big}x{L_big}", dtype="f64" if precision == 0 else "f32", bytes_per_site=6 * cplx,
                ms=t * 1e3, gbs=bytes_alg / t / 1e9)


def dslash_half_roofline(L_big: int = 4096, iters: int = 20):
    """The fine Wilson apply on half-precision storage with per-site norms (mg_dslash, MG_FP16) on a
    lattice far larger than L2: 32 algorithmic bytes per site (psi 8 + norm 4, U 8, out 8 + norm 4)."""
    import torch
    import paper_0707_4018_gb300 as mg
    V = L_big * L_big
    g = torch.Generator(device="cuda").manual_seed(5)
    ang = torch.rand((V, 2), device="cuda", generator=g, dtype=torch.float64) * 2 * np.pi
    U = torch.polar(torch.ones_like(ang), ang).to(torch.complex64)
    psi = torch.randn((V, 2), device="cuda", generator=g, dtype=torch.complex64)
    Uh, ph, oh = mg.half_links(V), mg.half_spinor(V), mg.half_spinor(V)
    mg.mg_half_convert(2, U, Uh, V)
    mg.mg_half_convert(0, psi, ph, V)
    del U, psi
    stream = torch.cuda.current_stream()
    for _ in range(3):
        mg.mg_dslash_half(Uh, ph, oh, 0.01, (L_big, L_big))
    ms = []
    for _ in range(iters):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mg.mg_dslash_half(Uh, ph, oh, 0.01, (L_big, L_big))
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms) * 1e-3
    return dict(lattice=f"{L_big}x{L_big}", dtype="f16 storage, f32 arithmetic", bytes_per_site=32, ms=t * 1e3,
                gbs=V * 32 / t / 1e9, sites_per_s=V / t)


def dslash4_roofline(precision: int, dims=(32, 32, 32, 64), iters: int = 20, compare_gather: bool = True):
    """4d SU(3) Wilson apply alone on a lattice far larger than L2 (32^3 x 64: 1 GB per FP32
    apply): algorithmic bytes / time. Links are Gaussian 3 x 3 matrices (the timing does not
    depend on the values; the parity tests use SU(3) fields)."""
    import torch
    import paper_0707_4018_gb300 as mg
    dt = torch.complex128 if precision == 0 else torch.complex64
    V = int(np.prod(dims))
    g = torch.Generator(device="cuda").manual_seed(6)
    U = torch.randn((V, 4, 3, 3), device="cuda", generator=g, dtype=dt) / 3.0
    psi = torch.randn((V, 4, 3), device="cuda", generator=g, dtype=dt)
    out = torch.empty_like(psi)
    stream = torch.cuda.current_stream()
    cplx = 16 if precision == 0 else 8
    per_site = (12 + 36 + 12) * cplx  # psi in, 4 links, psi out

    def timed():
        for _ in range(3):
            mg.mg_dslash(U, psi, out, 0.01, dims, precision)
        ms = []
        for _ in range(iters):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mg.mg_dslash(U, psi, out, 0.01, dims, precision)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms) * 1e-3

    t = timed()
    res = dict(lattice="x".join(str(v) for v in dims), dtype="f64" if precision == 0 else "f32",
               bytes_per_site=per_site, flop_per_site=1368, ms=t * 1e3, gbs=V * per_site / t / 1e9,
               tflops=V * 1368 / t / 1e12,
               kernel="dslash4_tile_kernel (8x2x2x2 tiles)" if precision == 1 else "dslash4_kernel<double>")
    if precision == 1 and compare_gather:
        # the warp-gather kernel on the same inputs
        os.environ["MG_DSLASH4_GATHER"] = "1"
        try:
            tg = timed()
        finally:
            del os.environ["MG_DSLASH4_GATHER"]
        res["warp_gather_kernel"] = dict(ms=tg * 1e3, gbs=V * per_site / tg / 1e9)
    return res


# several gauge configurations of uneven sizes, 16 sources each (workload id, L, beta)
MIX_FIELDS = ((0, 64, 6.0), (2, 128, 6.0), (1, 256, 6.0), (1, 256, 10.0))
MIX_RHS = 16
MIX_DM = 0.02


def mixed_sizes(precision: int = 1, reps: int = 2):
    """Solves/s including setup for a set of gauge configurations of uneven lattice sizes, each with
    MIX_RHS Gaussian sources at m = m_c + 0.02: per configuration one setup and one batched solve
    (mg_solve_batch, all sources in lockstep), the configurations concurrently (one host thread and
    context stream each). Fields without a stored m_c are skipped (and listed)."""
    import torch
    import paper_0707_4018_gb300 as mg
    table = mcrit_table()
    cfgs, skipped = [], []
    for wid, Lm, beta in MIX_FIELDS:
        row = table.get(f"w{wid}_L{Lm}_b{beta:g}")
        U, theta, _ = inputs.schwinger_links(Lm, beta, sweeps=2000, workload_id=wid)
        if row is None or row["theta_digest"] != inputs.field_digest(theta):
            skipped.append(f"{Lm}x{Lm} beta {beta:g}")
            continue
        seed = inputs.workload_seed(wid, Lm, beta)
        chi = np.stack([inputs.gaussian_source(Lm, Lm, seed=seed, index=10 + i) for i in range(MIX_RHS)])
        cfgs.append(dict(L=Lm, beta=beta, m=row["m_crit"] + MIX_DM, U=torch.from_numpy(U).cuda(),
                         chi=torch.from_numpy(chi).cuda(),
                         psi=torch.empty((MIX_RHS, Lm * Lm, 2), dtype=torch.complex128, device="cuda")))
    if not cfgs:
        return {"skipped": skipped}

    def params():
        p = mg_params(precision)
        p.max_rhs = MIX_RHS
        return p

    def one(cf, res):
        ctx = mg.Context.setup(cf["U"], cf["m"], (cf["L"], cf["L"]), params())
        st = ctx.solve_batch(cf["chi"], cf["psi"], TOL, raise_on_fail=False)
        ctx.close()
        res.append((cf["L"], cf["beta"], st))

    best = None
    for _ in range(reps):  # the first repetition also warms up (graph capture, pool)
        res = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=one, args=(cf, res)) for cf in cfgs]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if len(res) != len(cfgs):
            raise RuntimeError("a configuration of the mixed-size batch failed")
        if best is None or dt < best[0]:
            best = (dt, res)
    dt, res = best
    n = MIX_RHS * len(cfgs)
    return {"workload": "2d U(1) configurations of uneven sizes " + ", ".join(f"{c['L']}^2 beta {c['beta']:g}" for c in cfgs)
                        + f"; {MIX_RHS} Gaussian sources each at m_c + {MIX_DM}, 3-level MG, one batched solve per "
                        "configuration, the configurations concurrently",
            "solves": n, "seconds": dt, "solves_per_s_incl_setup": n / dt, "skipped": skipped,
            "iters_max": {f"{Lm}^2 b{beta:g}": max(s["iters"] for s in st) for Lm, beta, st in res},
            "converged": all(s["converged"] for _, _, st in res for s in st),
            "worst_true_rel_residual": max(s["true_rel_residual"] for _, _, st in res for s in st)}


SU3_DIMS = (16, 16, 16, 32)
SU3_RHS = 12


def su3_params(precision: int):
    """4d SU(3) hierarchy: two levels, 4^4 blocks, Nv = 24 split by chirality (48 coarse dofs),
    one relaxation pass of 400 MR iterations (deeper relaxation in place of adaptive passes,
    which lower the quality of well-relaxed 4d vectors, in the oracle too), MR 4 + 4, coarse
    GCR(64) to 0.3 with block Jacobi, at most 128 coarse iterations per cycle (near m_c an
    inexact coarse solve costs fewer operations than an exact one; the outer flexible GCR absorbs
    it), outer restart 32 (the 22-25 outer iterations then run without a restart). At m_c + 0.005
    these settings took 144 ms per solve and 0.47 s of setup, against 227 ms and 0.30 s with 200
    relaxation steps and a coarse tolerance of 0.05; the batch of 12 took 553 / 542 / 550 / 526 ms
    with outer restarts 16 / 8 / 12 / 24 (24-26 outer iterations, 22 with 24)."""
    import paper_0707_4018_gb300 as mg
    return mg.mg_default_params(levels=2, blocks=[(4, 4, 4, 4)], Nv=[24], precision=precision, chiral_split=1,
                                n_pass=1, nu_setup=400, coarsest_tol=0.3, coarsest_restart=64,
                                coarsest_max_iter=128, gcr_restart=32, max_iter=300, max_rhs=SU3_RHS)


def su3_workload(precisions=(1, 0), nrhs: int = SU3_RHS, batched: bool = True, singles: bool = True):
    """Solves/s including setup on the 4d SU(3) workload: APE-smeared links on 16^3 x 32, m = m_c + 0.005
    (m_c from the oracle's table when present, else m = 0), 12 Gaussian sources to 1e-10, one setup."""
    import torch
    import paper_0707_4018_gb300 as mg
    import inputs
    U = inputs.su3_links(SU3_DIMS, seed=inputs.workload_seed(3, SU3_DIMS[0], 0.0))
    row = mcrit_table().get("w3_su3_" + "x".join(str(v) for v in SU3_DIMS))
    m_ok = row is not None and row.get("links_digest") == inputs.field_digest(U)
    m = row["m_crit"] + 0.005 if m_ok else 0.0
    V = int(np.prod(SU3_DIMS))
    Ud = torch.from_numpy(U).cuda()
    chis = [torch.from_numpy(inputs.gaussian_spinor(V, 12, 15, k)).cuda() for k in range(nrhs)]
    psi = torch.empty((V, 12), dtype=torch.complex128, device="cuda")
    out = {"workload": "4d SU(3) Wilson-Dirac 16^3x32, DeGrand-Rossi, APE-smeared links (4 steps, alpha 0.5); "
                       "2-level MG 4^4 blocks, Nv=24 chirality-split (48x48 coarse blocks), 12 Gaussian sources, tol 1e-10",
           "m": m, "m_from": (f"m_c + 0.005, m_c from the oracle's Arnoldi scan of "
                              f"{row.get('m_crit_from', 'this field')}") if m_ok else "0.0 (no m_c in the table)"}
    for prec in precisions:
        if not singles:
            break
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = mg.Context.setup(Ud, m, SU3_DIMS, su3_params(prec))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sts = [ctx.solve(c, psi, TOL, raise_on_fail=False) for c in chis]
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ctx.close()
        out["mixed" if prec == 1 else "fp64"] = {
            "solves_per_s_incl_setup": nrhs / (t2 - t0), "solves_per_s_excl_setup": nrhs / (t2 - t1),
            "setup_s": t1 - t0, "ms_per_solve": (t2 - t1) / nrhs * 1e3, "iters": [st["iters"] for st in sts],
            "coarse_iters": [st["coarsest_iters"] for st in sts], "converged": all(st["converged"] for st in sts),
            "worst_true_rel_residual": max(st["true_rel_residual"] for st in sts)}
    if batched and 1 in precisions:
        # the same sources as one batch: lockstep solve, coarse operator on tensor cores
        prec = 1
        chi_b = torch.stack(chis)
        psi_b = torch.empty_like(chi_b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = mg.Context.setup(Ud, m, SU3_DIMS, su3_params(prec))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sts = ctx.solve_batch(chi_b, psi_b, TOL, raise_on_fail=False)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        ctx.close()
        out["mixed_batched"] = {
            "solves_per_s_incl_setup": nrhs / (t2 - t0), "solves_per_s_excl_setup": nrhs / (t2 - t1),
            "setup_s": t1 - t0, "ms_per_batch": (t2 - t1) * 1e3, "iters": [st["iters"] for st in sts],
            "coarse_iters_total": sts[0]["coarsest_iters"], "converged": all(st["converged"] for st in sts),
            "worst_true_rel_residual": max(st["true_rel_residual"] for st in sts)}
    return out


# the paper's own experiment: (stored field, lattice, workload id, blocks per coarsening)
PAPER_CASES = (("w0_L64_b6", 64, 0, [(4, 4)]), ("w2_L128_b6", 128, 2, [(8, 8)]),
               ("w2_L128_b6", 128, 2, [(4, 4), (4, 4)]))


def paper_mgcg(tol: float = 1e-14):
    """The paper's own experiment on the GPU (numerical-results section): plain CG against CG
    preconditioned by the adaptive V-cycle on the normal equations D^dagger D psi = D^dagger chi,
    beta = 6 thermal fields at m_hat = m - m_c = 0.01, point source, relative residual 1e-14; M = 8
    vectors, the frozen two-step MR smoother, exact coarsest solve; setup with 100 relaxation steps
    and 3 passes at the solve's mass. Cost in fine D^dagger D applications as the paper counts it
    (6 per MG-CG iteration). The 64^2 field has Q = 0 as in the paper's quoted case; the 128^2
    field of the recipe has Q = 9. Without smoothed aggregation (R7) the paper's three-level
    hierarchy (4 x 4 twice) converges much more slowly than two levels."""
    import torch
    import paper_0707_4018_gb300 as mg
    table = mcrit_table()
    out = {"paper": {"lattice": "128x128", "beta": 6, "m_hat": 0.01, "Q": 0, "cg_iters": 3808, "mgcg_iters": 26,
                     "fine_DdagD_per_mgcg_iter": 6, "hardware": "not stated"},
           "tol": tol, "runs": []}
    fields = {}
    for key, Lf, wid, blocks in PAPER_CASES:
        row = table[key]
        if key not in fields:
            (U, theta, _), = inputs.schwinger_links_gpu(Lf, 6.0, sweeps=2000, workload_id=wid)
            fields[key] = (torch.from_numpy(U).cuda(), inputs.field_digest(theta) == row["theta_digest"])
        Ud, digest_ok = fields[key]
        m = row["m_crit"] + 0.01
        p = mg.mg_default_params(levels=len(blocks) + 1, blocks=blocks, Nv=[8] * len(blocks), n_pass=3,
                                 nu_setup=100)
        chi = torch.zeros((Lf * Lf, 2), dtype=torch.complex128, device="cuda")
        chi[0, 0] = 1.0
        psi = torch.empty_like(chi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = mg.CgContext.setup(Ud, m, (Lf, Lf), p)
        setup_s = time.perf_counter() - t0
        st_mg = ctx.solve(chi, psi, tol, max_iter=20000, precondition=True, raise_on_fail=False)
        st_cg = ctx.solve(chi, psi, tol, max_iter=20000, precondition=False, raise_on_fail=False)
        ctx.close()
        out["runs"].append({
            "field": key, "lattice": f"{Lf}x{Lf}", "Q": row.get("Q"), "digest_ok": digest_ok, "m_hat": 0.01,
            "levels": len(blocks) + 1, "blocks": [list(b) for b in blocks], "setup_s": setup_s,
            "mgcg": {"iters": st_mg["iters"], "fine_DdagD_apps": st_mg["fine_apps"], "ms": st_mg["ms"],
                     "converged": st_mg["converged"], "rel_residual": st_mg["rel_residual"]},
            "cg": {"iters": st_cg["iters"], "fine_DdagD_apps": st_cg["fine_apps"], "ms": st_cg["ms"],
                   "converged": st_cg["converged"], "rel_residual": st_cg["rel_residual"]}})
    return out


def coarsest_flops(iters: int, restart: int, n: int) -> float:
    """Algorithmic flops of one GCR solve on the preconditioned coarsest stencil (N = 8).

    Iteration with basis index k: stencil 40 complex MACs per dof (320 n), k + 2 dot
    products (8 n each), projection of w and z (16 k n), x / r updates (16 n), scaling
    (16 n); each restart cycle ends with a true residual (322 n); plus |b|^2 (4 n) and
    the final x = M y (64 n).
    """
    f = 4.0 * n + 64.0 * n
    cycles = 0
    for i in range(iters):
        k = i % restart
        if k == 0:
            cycles += 1
        f += n * (320 + 8 * (k + 2) + 16 * k + 32)
    return f + max(cycles, 1) * 322.0 * n


CLUSTER_CTAS = 16   # CTAs (one per SM) of the coarsest solve's thread-block cluster
GPU_SMS = 152
# DRAM bytes per launch of coarsest_gcr_cluster_kernel (ncu, profiles/coarsest_gcr_cluster_256x256.md)
CLUSTER_DRAM_BYTES = 3873536


def coarsest_roofline(fields, iters_rep: int = 20):
    """Live timing of the dominant kernel of the step, the coarsest GCR on one 16-CTA cluster (the
    bench's mixed-precision hierarchy of the beta = 6 field: 32^2 coarse sites x 8 = 8192 dofs), with
    its arithmetic (FP32 operator and Krylov vectors, FP64 cross-CTA sums) against the FP32 FMA rate
    measured in this process."""
    import torch
    import paper_0707_4018_gb300 as mg
    f = [f for f in fields if f["beta"] == 6.0][0]
    ctx = mg.Context.setup(f["U_dev"], f["m_c"] + DMS[0], (L, L), mg_params(mg.MG_FP32))
    n_sites, n_int = ctx.level_size(2)
    g = torch.Generator(device="cuda").manual_seed(11)
    b = torch.randn((n_sites, n_int), dtype=torch.complex128, device="cuda", generator=g)
    x = torch.empty_like(b)
    for _ in range(3):
        ctx.coarsest_solve(b, x)
    ms, flops = [], []
    for _ in range(iters_rep):
        it, t = ctx.coarsest_solve(b, x)
        ms.append(t)
        flops.append(coarsest_flops(it, int(ctx.params.coarsest_restart), n_sites * n_int))
    ctx.close()
    t = statistics.median(ms) * 1e-3
    peak32 = mg.mg_alu_peak(1)
    peak64 = mg.mg_alu_peak(0)
    return dict(kernel="coarsest_gcr_cluster_kernel (coarsest GCR on one 16-CTA cluster, 32x32 coarse sites x 8, "
                       "FP32 operator and vectors, FP64 sums)",
                iters=it, ms=t * 1e3, tflops=statistics.median(flops) / t / 1e12, peak_fp32=peak32,
                peak_fp64=peak64)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def cpu_baseline(budget_s: float | None = 25.0, threads: int | None = None, solutions: dict | None = None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload: beta = 6 only,
    adaptive setup at the lightest mass then solves at the three masses (the GPU step's
    amortisation: 3 solves per setup) until the budget (None: all three). threads: BLAS
    threads (None: all host cores; numpy's elementwise work is single-threaded either way).
    solutions: when a dict, receives the oracle's psi per mass index (the parity reference of
    the GPU's beta = 6 results)."""
    import contextlib
    try:
        import threadpoolctl
        limit = threadpoolctl.threadpool_limits(threads) if threads else contextlib.nullcontext()
    except ImportError:
        limit = contextlib.nullcontext()
    with limit:
        return _cpu_baseline(budget_s, threads, solutions)


def _cpu_baseline(budget_s, threads, solutions=None):
    from oracle import setup as osetup, solvers as osolvers
    from oracle.lattice import Lattice
    table = mcrit_table()
    beta = 6.0
    U, _, _ = inputs.schwinger_links(L, beta, sweeps=2000, workload_id=WORKLOAD_ID)
    mc = table[f"w{WORKLOAD_ID}_L{L}_b{beta:g}"]["m_crit"]
    lat = Lattice((L, L))
    p = osetup.MGParams(levels=3, blocks=((4, 4), (2, 2)), Nv=(8, 8), coarsest_tol=0.2, coarsest_restart=16,
                        coarsest_lu_max=2048)
    seed = inputs.workload_seed(WORKLOAD_ID, L, beta)
    t0 = time.perf_counter()
    hier = osetup.adaptive_setup(U, mc + DMS[0], lat, p)
    solves = 0
    for i, dm in enumerate(DMS):
        if i > 0:
            osetup.update_mass(hier, mc + dm)
        chi = inputs.gaussian_source(L, L, seed=seed, index=i)
        x, _ = osolvers.mg_solve(hier, chi, TOL)
        if solutions is not None:
            solutions[i] = x
        solves += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    if threads:
        cores = threads
    else:
        try:
            import threadpoolctl
            cores = max(info.get("num_threads", 1) for info in threadpoolctl.threadpool_info()) or 1
        except Exception:
            cores = os.cpu_count() or 1
    return dict(value=solves / dt, unit="solves/s", cores=cores, kind="oracle", seconds=dt, solves=solves,
                sample=f"beta=6 only: oracle setup at m_c+0.005 then {solves} solve(s) "
                       f"(of the 9-solve step), 256x256, tol 1e-10")


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; independent solves per rank)
# ---------------------------------------------------------------------------
def init_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return dist


def barrier(d):
    if d is not None:
        d.barrier()


def max_over_ranks(x: float, d) -> float:
    if d is None:
        return x
    import torch
    dev = "cuda" if d.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, d) -> float:
    if d is None:
        return x
    import torch
    dev = "cuda" if d.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    d.all_reduce(t, op=d.ReduceOp.SUM)
    return float(t.item())


def rank_of(d) -> int:
    return 0 if d is None else d.get_rank()


def world_of(d) -> int:
    return 1 if d is None else d.get_world_size()


def run_reference(args, d):
    """The oracle arm: the FP64 CPU oracle timed on the host cores (rank 0 only)."""
    if rank_of(d) != 0:
        return
    # each step: one oracle setup and its three solves (the GPU step's amortisation of 3 solves per
    # setup, for beta = 6); steps run until about 150 s have passed (at least one), so the arm
    # ends within a few minutes whatever --steps is
    per_step = []
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        per_step.append(cpu_baseline(budget_s=None))
        if time.perf_counter() - t0 > 150.0:
            break
    solves = sum(c["solves"] for c in per_step)
    secs = sum(c["seconds"] for c in per_step)
    v = solves / secs
    sample = (f"{len(per_step)} of {args.steps} step(s) timed; each: " + per_step[0]["sample"])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": f"{L}x{L}", "betas": list(BETAS), "m_minus_mc": list(DMS),
                       "tol": TOL},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": per_step[0]["cores"], "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_only(case: str):
    """Small fixed cases for profiler captures (no timing claims are made from them)."""
    import torch
    import paper_0707_4018_gb300 as mg
    mg.load()
    if case == "su3":
        print(json.dumps({"case": case, **su3_workload()}))
        return
    if case == "mixed-sizes":
        print(json.dumps({"case": case, **mixed_sizes()}))
        return
    if case == "config2":
        print(json.dumps({"case": case, **config2_batch()}))
        return
    if case == "paper":
        print(json.dumps({"case": case, **paper_mgcg()}))
        return
    if case == "learned":
        print(json.dumps({"case": case, **learned_setup_eval()}))
        return
    if case == "large":
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        print(json.dumps({"case": case, **config1_large(flush)}))
        return
    if case == "su3-batch-prof":  # mixed precision, setup and one batch of 12 sources (launch-list profiling)
        r = su3_workload((1,), SU3_RHS, batched=True, singles=False)
        print(json.dumps({"case": case, **r}))
        return
    if case == "su3-prof":  # mixed precision, setup and 2 solves (launch-list profiling)
        print(json.dumps({"case": case, **su3_workload((1,), 2, batched=False)}))
        return
    if case == "dslash4-sweep":
        # the FP32 4d apply on 32^3 x 64 with each kernel variant (tile shapes, warp gather)
        res = {}
        for name, env in (("gather", ("MG_DSLASH4_GATHER", "1")), ("tileA_8x4x4x4", ("MG_DSLASH4_TILE", "0")),
                          ("tileB_8x4x4x2", ("MG_DSLASH4_TILE", "1")), ("tileC_4x4x4x2", ("MG_DSLASH4_TILE", "2")),
                          ("tileD_8x4x2x2", ("MG_DSLASH4_TILE", "3")), ("tileB_3cta", ("MG_DSLASH4_TILE", "4")),
                          ("tileC_6cta", ("MG_DSLASH4_TILE", "5")), ("tileE_4x4x2x2", ("MG_DSLASH4_TILE", "6")),
                          ("tileF_8x2x2x2", ("MG_DSLASH4_TILE", "7"))):
            os.environ[env[0]] = env[1]
            try:
                r = dslash4_roofline(1, iters=10, compare_gather=False)
            finally:
                del os.environ[env[0]]
            res[name] = {"ms": r["ms"], "gbs": r["gbs"]}
        print(json.dumps({"case": case, **res}))
        return
    if case.startswith("dslash4"):
        r = dslash4_roofline(1 if case == "dslash4-f32" else 0, iters=3, compare_gather=False)
        print(json.dumps({"case": case, **r}))
        return
    if case == "dslash-f16":
        print(json.dumps({"case": case, **dslash_half_roofline(iters=3)}))
        return
    if case.startswith("dslash"):
        r = dslash_roofline(1 if case == "dslash-f32" else 0, iters=3)
        print(json.dumps({"case": case, **r}))
        return
    if case == "coarse-tc":
        # level 1 of the 256^2 hierarchy (64^2 coarse sites x 8) applied to 16 vectors
        U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=2000, workload_id=WORKLOAD_ID)
        ctx = mg.Context.setup(torch.from_numpy(U).cuda(), 0.1, (L, L), mg_params(mg.MG_FP32))
        n_sites, n_int = ctx.level_size(1)
        R = 16
        g = torch.Generator(device="cuda").manual_seed(9)
        x = torch.randn((R, n_sites, n_int), dtype=torch.complex64, device="cuda", generator=g)
        y = torch.empty_like(x)
        res = {}
        stream = torch.cuda.current_stream()
        for tc in (True, False):
            for _ in range(3):
                ctx.coarse_apply_mrhs(1, x, y, tc)
            ms = []
            for _ in range(20):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.coarse_apply_mrhs(1, x, y, tc)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            t = statistics.median(ms) * 1e-3
            res["tensor" if tc else "cuda_core"] = {"us_per_call_incl_sync": t * 1e6,
                                                    "gflops": 2560 * R * n_sites / t / 1e9}
        print(json.dumps({"case": case, "coarse_sites": n_sites, "rhs": R, **res, "autotune": mg.autotune_report()}))
        ctx.close()
        return
    if case == "coarse-tc4":
        # the 4d coarse level of the 16^3 x 32 hierarchy (512 sites x 48) on 12 and 16 vectors
        import inputs as inp
        U4 = inp.su3_links(SU3_DIMS, seed=inp.workload_seed(3, SU3_DIMS[0], 0.0))
        p4 = su3_params(mg.MG_FP32)
        p4.nu_setup = 20
        ctx = mg.Context.setup(torch.from_numpy(U4).cuda(), 0.0, SU3_DIMS, p4)
        n_sites, n_int = ctx.level_size(1)
        stream = torch.cuda.current_stream()
        out = {"case": case, "coarse_sites": n_sites, "n_int": n_int}
        for R in (12, 16):
            g = torch.Generator(device="cuda").manual_seed(9)
            x = torch.randn((R, n_sites, n_int), dtype=torch.complex64, device="cuda", generator=g)
            y = torch.empty_like(x)
            for tc in (1, 2, 3, 0):  # BF16 operands, split vectors, split vectors and operator, CUDA cores
                for _ in range(3):
                    ctx.coarse_apply_mrhs(1, x, y, tc)
                ms = []
                for _ in range(20):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ctx.coarse_apply_mrhs(1, x, y, tc)
                    e1.record(stream)
                    e1.synchronize()
                    ms.append(e0.elapsed_time(e1))
                t = statistics.median(ms) * 1e-3
                name = {0: "cuda_core", 1: "tensor", 2: "tensor_split_vectors", 3: "tensor_split_both"}[tc]
                out[f"{name}_rhs{R}"] = {
                    "us_per_call_incl_sync": t * 1e6, "gflops": 9 * 48 * 48 * 8 * R * n_sites / t / 1e9}
        print(json.dumps(out))
        ctx.close()
        return
    if case == "transfer":
        Lt = 1024
        p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=mg.MG_FP32, n_pass=1,
                                 nu_setup=4, coarsest_tol=0.2)
        ctx = mg.Context.setup(torch.from_numpy(inputs.hot_links(Lt, Lt, seed=3)).cuda(), 0.1, (Lt, Lt), p)
        r = torch.from_numpy(inputs.gaussian_source(Lt, Lt, seed=4)).cuda()
        z = torch.empty_like(r)
        for _ in range(5):
            ctx.vcycle(r, z)
        torch.cuda.synchronize()
        print(json.dumps({"case": case, "lattice": f"{Lt}x{Lt}", "cycles": 5}))
        ctx.close()
        return
    if case == "step":
        # one step of the headline workload (3 setups, 9 solves), the launch list's sample
        fdev = device_fields(make_inputs(0))
        stats = []
        run_step(fdev, mg.MG_FP32, stats_out=stats)
        torch.cuda.synchronize()
        print(json.dumps({"case": case, "mode": STEP_MODE, "iters": [s["iters"] for s in stats]}))
        return
    beta = 6.0
    U, _, _ = inputs.schwinger_links(L, beta, sweeps=2000, workload_id=WORKLOAD_ID)
    mc = mcrit_table()[f"w{WORKLOAD_ID}_L{L}_b{beta:g}"]["m_crit"]
    seed = inputs.workload_seed(WORKLOAD_ID, L, beta)
    if case == "vcycle":
        # the preconditioner alone: 5 warm-up cycles, then 20 replays of the captured graph
        ctx = mg.Context.setup(torch.from_numpy(U).cuda(), mc + DMS[0], (L, L), mg_params(mg.MG_FP32))
        r = torch.from_numpy(inputs.gaussian_source(L, L, seed=seed)).cuda()
        z = torch.empty_like(r)
        for _ in range(5):
            ctx.vcycle(r, z)
        torch.cuda.synchronize()
        n0 = mg.mg_kernel_launches()
        t0 = time.perf_counter()
        for _ in range(20):
            ctx.vcycle(r, z)
        torch.cuda.synchronize()
        print(json.dumps({"case": case, "us_per_cycle_host_clock": (time.perf_counter() - t0) / 20 * 1e6,
                          "launches_per_cycle": (mg.mg_kernel_launches() - n0) / 20}))
        ctx.close()
        return
    fd = dict(beta=beta, m_c=mc, U_dev=torch.from_numpy(U).cuda(),
              chi_dev=[torch.from_numpy(inputs.gaussian_source(L, L, seed=seed, index=i)).cuda() for i in range(3)],
              psi_dev=[torch.empty((L * L, 2), dtype=torch.complex128, device="cuda") for _ in DMS])
    stats = []
    run_step([fd], mg.MG_FP32, stats_out=stats)
    print(json.dumps({"case": case, "iters": [s["iters"] for s in stats]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-fp16", action="store_true")
    ap.add_argument("--serial", action="store_true", help="run the betas of a step one after another")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 1024^2 sweep points")
    ap.add_argument("--threads", action="store_true",
                    help="solve with one host thread and host-driven loop per solve instead of one graph launch")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned near-null setup evaluation")
    ap.add_argument("--no-config2", action="store_true", help="skip the many-configuration x many-source batch")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's MG-CG experiment")
    ap.add_argument("--only", default=None, choices=["paper", "step", "dslash4-sweep", "dslash-f16", "dslash-f32", "dslash-f64", "dslash4-f32", "dslash4-f64", "solve", "vcycle",
                                                      "transfer", "coarse-tc", "coarse-tc4", "su3", "su3-prof",
                                                      "su3-batch-prof", "mixed-sizes", "learned", "large",
                                                      "config2"],
                    help="profiling cases: the Dslash timing loop alone (2d, or 4d SU(3)), one beta's setup + 3 solves, "
                         "25 mixed-precision V-cycles after one beta's setup, or 5 V-cycles on a 1024^2 "
                         "hierarchy (fine level larger than L2, for the restriction and prolongation), or the "
                         "level-1 coarse apply on 16 vectors, tensor cores and CUDA cores")
    args = ap.parse_args()
    global CONCURRENT, STEP_MODE
    CONCURRENT = not args.serial
    STEP_MODE = "threads" if args.threads else "graph"
    if args.warmup < 3:
        raise SystemExit("warmup must be >= 3")
    if args.only is not None:
        run_only(args.only)
        return
    d = init_dist()
    if args.impl == "reference":
        run_reference(args, d)
        return
    import torch
    import paper_0707_4018_gb300 as mg
    rank = rank_of(d)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    mg.load()
    fields = make_inputs(rank)
    fields_dev = device_fields(fields)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    sampler = ClockSampler(local)
    mixed = timed_steps(fields_dev, mg.MG_FP32, args.steps, args.warmup, flush, d, sampler=sampler)
    total_solves = sum_over_ranks(mixed["solves"], d)
    value = total_solves / (mixed["ms"] * 1e-3)
    worst_res = max(s["true_rel_residual"] for s in mixed["stats"])
    iters = [s["iters"] for s in mixed["stats"]]

    mixed_sols = [[p.clone() for p in f["psi_dev"]] for f in fields_dev]
    fp16 = None
    fp16_sols = None
    if not args.no_fp16:
        r = timed_steps(fields_dev, mg.MG_FP16, args.steps, 3, flush, d)
        fp16_sols = [[p.clone() for p in f["psi_dev"]] for f in fields_dev]
        fp16 = dict(value=sum_over_ranks(r["solves"], d) / (r["ms"] * 1e-3), unit="solves/s",
                    ms_per_step=r["ms"] / args.steps, iters=[s["iters"] for s in r["stats"]],
                    worst_true_rel_residual=max(s["true_rel_residual"] for s in r["stats"]),
                    precision="FP64 outer GCR, FP32 V-cycle whose fine level stores links and the MR vectors "
                              "r, A r in FP16 with per-site FP32 norms")
    fp64 = None
    if not args.no_fp64:
        r = timed_steps(fields_dev, mg.MG_FP64, args.steps, 3, flush, d)
        fp64 = dict(value=sum_over_ranks(r["solves"], d) / (r["ms"] * 1e-3), unit="solves/s",
                    ms_per_step=r["ms"] / args.steps, iters=[s["iters"] for s in r["stats"]],
                    worst_true_rel_residual=max(s["true_rel_residual"] for s in r["stats"]),
                    mixed_vs_fp64_rel_diff=solution_diffs(mixed_sols, [f["psi_dev"] for f in fields_dev]))
        if fp16_sols is not None:
            fp64["fp16_vs_fp64_rel_diff"] = solution_diffs(fp16_sols, [f["psi_dev"] for f in fields_dev])
    fp64_sols = [[p.clone() for p in f["psi_dev"]] for f in fields_dev] if fp64 is not None else None

    e2e = None
    if not args.no_e2e:
        host_out = {f["beta"]: [torch.empty((L * L, 2), dtype=torch.complex128).pin_memory() for _ in DMS]
                    for f in fields_dev}
        r = timed_steps(fields_dev, mg.MG_FP32, args.steps, 3, flush, d, host_io=host_out)
        h2d = sum(f["U_host"].numel() * 16 + sum(c.numel() * 16 for c in f["chi_host"]) for f in fields_dev)
        d2h = sum(len(DMS) * L * L * 2 * 16 for _ in fields_dev)
        e2e = dict(value=sum_over_ranks(r["solves"], d) / (r["ms"] * 1e-3), unit="solves/s",
                   h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h)

    peak, peak_kind = measured_peaks()
    ds32 = dslash_roofline(1)
    ds64 = dslash_roofline(0)
    ds4 = dslash4_roofline(1)
    ds16 = dslash_half_roofline()
    su3 = su3_workload() if world_of(d) == 1 or rank == 0 else None
    mix = mixed_sizes() if world_of(d) == 1 or rank == 0 else None
    cr = coarsest_roofline(fields_dev)
    large = config1_large(flush) if (world_of(d) == 1 or rank == 0) and not args.no_large else None
    learned = learned_setup_eval() if (world_of(d) == 1 or rank == 0) and not args.no_learned else None
    many = config2_batch() if (world_of(d) == 1 or rank == 0) and not args.no_config2 else None
    paper = paper_mgcg() if (world_of(d) == 1 or rank == 0) and not args.no_paper else None

    cpu = None
    if rank == 0 and world_of(d) == 1 and not args.no_cpu:
        oracle_psi = {}
        cpu = cpu_baseline(solutions=oracle_psi)
        # the error of each beta = 6 result against the oracle's FP64 solve of the same system
        b6 = [i for i, f in enumerate(fields_dev) if f["beta"] == 6.0][0]
        err = {}
        for name, sols in (("mixed", mixed_sols), ("fp16", fp16_sols), ("fp64", fp64_sols)):
            if sols is not None:
                err[name] = {f"m_c+{DMS[i]:g}": float(np.linalg.norm(sols[b6][i].cpu().numpy() - x) /
                                                      np.linalg.norm(x)) for i, x in oracle_psi.items()}
        cpu["gpu_vs_oracle_rel_err_beta6"] = err
        one = cpu_baseline(budget_s=10.0, threads=1)
        cpu["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "seconds", "sample")}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world_of(d), "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mixed["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": f"{L}x{L}", "betas": list(BETAS), "m_minus_mc": list(DMS),
                   "solves_per_step": len(BETAS) * len(DMS), "precision": "FP64 outer GCR, FP32 V-cycle",
                   "l2": "flushed before every timed step (512 MiB write)", "tol": TOL,
                   "betas_run": ("concurrently: one host thread per beta runs its setup, two clones of it "
                                 "(Galerkin rebuilt per mass) and one multi-solve graph launch of its three solves "
                                 "(device-driven outer loops)" if STEP_MODE == "graph" else
                                 "concurrently: one host thread and context stream per beta and, through clones of "
                                 "the beta's setup (Galerkin rebuilt per mass), per mass (host-driven outer loops)")
                   if CONCURRENT else "one after another",
                   "gauge_digest_matches_table": all(f["digest_ok"] for f in fields) if rank == 0 else None},
        "solver": {"iters": iters, "worst_true_rel_residual": worst_res},
        "fp64_mg": fp64,
        "fp16_mg": fp16,
        "e2e": e2e,
        "gpu_launches": mixed["launches"],
        "clocks": mixed["clocks"],
        "roofline": {"bound": "alu", "kernel": cr["kernel"], "achieved": cr["tflops"], "peak": cr["peak_fp32"],
                     "unit": "TFLOP/s", "frac": cr["tflops"] / cr["peak_fp32"], "traffic": CLUSTER_DRAM_BYTES,
                     "traffic_source": "profiles/coarsest_gcr_cluster_256x256.md",
                     "ms_per_launch": cr["ms"], "iters_per_launch": cr["iters"],
                     "peak_kind": "measured in this run (mg_alu_peak: FP32 FMA loop over all SMs)",
                     "sms_used": CLUSTER_CTAS,
                     "frac_of_its_sms": cr["tflops"] / (cr["peak_fp32"] * CLUSTER_CTAS / GPU_SMS),
                     "fp64_peak_measured": cr["peak_fp64"],
                     "note": "latency-bound: 3 cluster barriers per GCR iteration on n = 8192; the kernel holds "
                             "16 of 152 SMs so the other solves of the step run beside it"},
        "dslash_hbm": {"f32": ds32, "f64": ds64, "peak_gbs": peak, "peak_kind": peak_kind,
                       "frac_f32": ds32["gbs"] / peak,
                       "traffic_f32": 780606208, "traffic_source": "profiles/dslash_f32_4096x4096.md",
                       "su3_4d_f32": {**ds4, "frac": ds4["gbs"] / peak},
                       "f16": {**ds16, "frac": ds16["gbs"] / peak}},
        "cpu_baseline": cpu,
        "su3_4d": su3,
        "mixed_sizes": mix,
        "config1_1024": large,
        "learned_setup": learned,
        "config2_many_configs": many,
        "paper_mgcg": paper,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
