#!/usr/bin/env python
"""Throughput of the plane-wave DFT energy + force evaluation (the call every DE
candidate and relaxation step of the paper makes, Sec. II A-D).

Workload: the 64-member DE population (cells of 8-32 Z_val=4 atoms, volume
135 bohr^3/atom +-20%, Ecut 12 Ha, FD kT 0.01 Ha; uneven plane-wave counts), one
step = one batched, cold-start, mixed-precision energy+force evaluation of all 64
members through the C ABI.  Metric: evaluations/s.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints ONE JSON line on rank 0.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload (the smallest member, one evaluation per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DFT energy+force evals/s (batched, mixed prec) vs plain FP64, ≤1e-5 Ha/atom"
WORKLOAD = "de_population_64"
MEMBERS = 64
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP32 CUDA-core peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes (read + write) per launch of the plane pass (k_plane_vpsi_ms) on this workload, the
# mean of one launch of each size class of one sub-batch (ncu capture, cold cache):
# (9.22 + 0.00 + 82.07 + 16.00) / 2 MB.  Set to None whenever the kernel changes after the capture.
PLANE_VPSI_TRAFFIC = (9.224e6 + 82.074e6 + 15.996e6) / 2


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _population(rank):
    """Weak scaling: rank r evaluates its own 64 members, candidates 64 r .. 64 r + 63."""
    import workloads
    return workloads.de_population(MEMBERS, start=MEMBERS * rank)


def _max_over_ranks(value, device=None):
    """Max of a per-rank float over the process group (the step time of the slowest rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _smallest(pop):
    return min(range(len(pop)), key=lambda i: (pop[i].natoms, i))


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def _oracle_eval(st):
    import oracle
    t = time.perf_counter()
    r = oracle.scf(st)
    return time.perf_counter() - t, r


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    pop = _population(0)
    i = _smallest(pop)
    st = pop[i]
    for _ in range(args.warmup):
        _oracle_eval(st)
    times = []
    for _ in range(args.steps):
        dt, _ = _oracle_eval(st)
        times.append(dt)
    total = sum(times)
    value = args.steps / total
    sample = f"member {i} ({st.natoms} atoms) of the population, one oracle evaluation per step"
    line = dict(metric=METRIC, value=value, unit="evals/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * total / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, members=MEMBERS, sample=sample, precision="fp64 (CPU oracle)"),
                cpu_baseline=dict(value=value, unit="evals/s", cores=_cores(), kind="oracle", sample=sample),
                e2e=dict(value=value, unit="evals/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        mhz, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                mhz.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not mhz:
            return None
        return dict(sm_mhz=float(np.median(mhz)), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(mhz))


_SCF = {}


def _tols(prec, st):
    """SCF stopping rule: FP64 path |dF| < 1e-8 Ha and residual < 1e-7; mixed path (FP32
    noise floor) |dF| < 1e-7 Ha per atom and residual < 1e-5 -- far inside 1e-5 Ha/atom."""
    if prec == "mixed":
        return dict(scf_tol_e=1e-7 * st.natoms, scf_tol_rho=1e-5, **_SCF)
    return dict(scf_tol_e=1e-8, scf_tol_rho=1e-7, **_SCF)


def _peaks():
    try:
        with open(MEASURED) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _warm_steps(args, sgo, batch, ctxs, pop, pos_host, pos_dev, e_dev, f_dev, s_dev, stream):
    """The relaxation regime: every member restarts from its previous density and
    wavefunctions after its atoms moved by a seeded 0.02 bohr Gaussian displacement (a
    relaxation step), one batched evaluation per step.  The positions of each step are
    copied to the device outside the timed region."""
    import torch
    rng = np.random.default_rng(77)
    for c in ctxs:
        c.set_warm(True)
    cur = [p.copy() for p in pos_host]
    ms, iters, ok = 0.0, [], 0
    for _ in range(args.steps):
        cur = [p + rng.normal(scale=0.02, size=p.shape) for p in cur]
        pos_dev.copy_(torch.from_numpy(np.concatenate([p.reshape(-1) for p in cur])))
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batch.energy_forces_device(pos_dev.data_ptr(), e_dev.data_ptr(), f_dev.data_ptr(), s_dev.data_ptr())
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
        iters += [c.info()["n_iter"] for c in ctxs]
        ok += int(np.sum(s_dev.cpu().numpy() == 0))
    for c in ctxs:
        c.set_warm(False)
    return dict(value=MEMBERS * args.steps / (ms / 1e3), unit="evals/s", steps=args.steps,
                start="previous density and wavefunctions, atoms moved by 0.02 bohr (Gaussian)",
                converged=f"{ok}/{MEMBERS * args.steps}",
                scf_iterations=dict(mean=float(np.mean(iters)), max=int(np.max(iters))))


RELAX_FMAX = 0.02 / 51.42208619083232   # 0.02 eV/Angstrom in Ha/bohr (Sec. II C's loose criterion)


def _relax_population(sgo, batch, ctxs, pop, max_rounds=60, method="pcg"):
    """Local relaxation (Sec. II C) of every member with the PCG driver (force-fitted
    preconditioner) over warm-started batched evaluations (sgo_relax_batch).  Every round
    evaluates the whole batch once."""
    drivers = [sgo.Relax(st.cell, st.pos, method=method, fmax=RELAX_FMAX, max_evals=max_rounds) for st in pop]
    t0 = time.perf_counter()
    rounds, status = batch.relax(drivers, max_rounds=max_rounds)
    dt = time.perf_counter() - t0
    info = [d.info() for d in drivers]
    evals = np.array([x["evals"] for x in info])
    conv = sum(1 for x in info if x["state"] == 1)
    names = dict(pcg="pcg (force-fitted inverse-Hessian preconditioner)", cg="cg", bfgs="bfgs")
    return dict(method=names[method], fmax_ha_bohr=RELAX_FMAX,
                rounds=int(rounds), seconds=dt, converged=f"{conv}/{len(pop)}",
                evals_per_member=dict(mean=float(evals.mean()), max=int(evals.max())),
                batched_evals_per_s=len(pop) * rounds / dt, member_status_ok=int(np.sum(status == 0)),
                start="the population's initial positions, warm-started from the previous runs' states")


def _de_search(sgo, generations=2, max_rounds=40):
    """Global search (Sec. II B) on the GPU: a population of 8 structures of 8 atoms in
    the diamond8 cell, relaxed (PCG, fmax 0.02 eV/A), then DE generations (triangle
    mutation, random plane/sphere cut-and-splice, relaxation of the children, greedy
    selection) with seeded random numbers."""
    import workloads
    pop_st = workloads.de_search_population(8, 8)
    base = pop_st[0]
    ctxs = [sgo.Context(st, precision="mixed", **_tols("mixed", st)) for st in pop_st]
    b = sgo.Batch(ctxs)
    drivers = [sgo.Relax(st.cell, st.pos, method="pcg", fmax=RELAX_FMAX, max_evals=max_rounds) for st in pop_st]
    t0 = time.perf_counter()
    b.relax(drivers, max_rounds=max_rounds)
    t_init = time.perf_counter() - t0
    best = [d.best() for d in drivers]
    f = np.array([e for e, _ in best])
    pop = np.array([x for _, x in best])
    rng = np.random.default_rng(6000)
    species = np.zeros(base.natoms, np.int32)
    gens = []
    for g in range(generations):
        u = rng.uniform(size=(len(f), sgo.DE_RANDOMS))
        t0 = time.perf_counter()
        pop, f, rep, cf = b.de_generation(base.cell, species, pop, f, u, max_rounds=max_rounds, fmax=RELAX_FMAX,
                                          max_evals=max_rounds)
        gens.append(dict(seconds=time.perf_counter() - t0, replaced=int(rep.sum()),
                         best_per_atom=float(f.min() / base.natoms)))
    return dict(population=f"8 x {base.natoms} atoms, {base.fft[0]}^3 grid, Ecut {base.ecut} Ha",
                relax="pcg, fmax 0.02 eV/A, <= %d batched evaluations per relaxation" % max_rounds,
                initial_relaxation_seconds=t_init, generations=gens)


def _ledger(sgo, st, prec, ref, i):
    """Errors of one member against the oracle: every eigenvalue and occupation, every
    energy term, the free energy and every force component (fresh single evaluation)."""
    ctx = sgo.Context(st, precision=prec, **_tols(prec, st))
    Fg, fg = ctx.energy_forces()
    eig, occ = ctx.eigen()
    t = ctx.terms()
    names = dict(kinetic="kinetic", nonlocal_="nonlocal", local="local", hartree="hartree", xc="xc",
                 ewald="ewald", minus_ts="minus_ts")
    return dict(member=i, natoms=st.natoms, nbands=st.nbands,
                eig_max_abs=float(np.max(np.abs(eig - ref.eig))),
                eig_occupied_max_abs=float(np.max(np.abs(eig - ref.eig)[ref.occ > 1e-3])),
                occ_max_abs=float(np.max(np.abs(occ - ref.occ))),
                terms_abs={k: float(abs(t[v] - ref.terms[k])) for k, v in names.items()},
                free_energy_per_atom=float(abs(Fg - ref.free_energy) / st.natoms),
                force_max_abs=float(np.max(np.abs(fg - ref.forces))),
                force_rms=float(np.sqrt(np.mean((fg - ref.forces) ** 2))))


def run_ours(args):
    import torch
    import paper_1603_02732_gb300 as sgo
    from paper_1603_02732_gb300 import build

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    sgo.load_library()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    pop = _population(rank)
    prec = args.precision
    ctxs = [sgo.Context(st, precision=prec, sub_batches=args.sub_batches, **_tols(prec, st)) for st in pop]
    batch = sgo.Batch(ctxs)
    pos_host = [np.ascontiguousarray(st.pos, dtype=np.float64) for st in pop]
    pos_dev = torch.tensor(np.concatenate([p.reshape(-1) for p in pos_host]), dtype=torch.float64, device=dev)
    e_dev = torch.zeros(MEMBERS, dtype=torch.float64, device=dev)
    f_dev = torch.zeros_like(pos_dev)
    s_dev = torch.zeros(MEMBERS, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step_device():
        batch.energy_forces_device(pos_dev.data_ptr(), e_dev.data_ptr(), f_dev.data_ptr(), s_dev.data_ptr())

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()

    def timed_steps():
        ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step_device()
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
        return ms

    # timed region: the default path (graph-driven SCF loop, sub-batches overlapped)
    batch.launches()
    clocks = Clocks(local)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms = timed_steps()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = batch.launches() // max(args.steps, 1)
    # the same steps again with the live kernel timer: CUDA events around every launch of
    # the timed kernel class need the host-driven loop (sub-batches one after another)
    batch.timer(args.kernel)
    timer_ms = timed_steps()
    kt = batch.timer_read()
    batch.timer(None)
    if ws > 1:
        import torch.distributed as dist
        total_ms = _max_over_ranks(total_ms, dev)
        timer_ms = _max_over_ranks(timer_ms, dev)
        dist.barrier()
    status = s_dev.cpu().numpy()
    iters = [c.info()["n_iter"] for c in ctxs]
    cstats = [c.stats() for c in ctxs]
    sweeps = [c["jacobi_sweeps"] for c in cstats]
    n_ok = int(np.sum(status == 0))
    value = ws * MEMBERS * args.steps / (total_ms / 1e3)

    # end to end through the host-pointer C-ABI call (H2D positions, D2H energies + forces)
    h2d = int(sum(p.nbytes for p in pos_host))
    d2h = int(MEMBERS * 8 + sum(p.nbytes for p in pos_host) + MEMBERS * 4)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        E, F, st = batch.energy_forces(pos_host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = ws * MEMBERS * e2e_steps / e2e_s

    out = None
    if rank == 0:
        peaks, src = _peaks()
        kname = args.kernel
        ach_tflops = kt["flops"] / (kt["ms"] / 1e3) / 1e12 if kt["ms"] > 0 else 0.0
        ach_gbs = kt["bytes"] / (kt["ms"] / 1e3) / 1e9 if kt["ms"] > 0 else 0.0
        roofline = dict(kernel=kname, bound="alu", achieved=ach_tflops, peak=FP32_PEAK_TFLOPS, unit="TFLOP/s",
                        frac=ach_tflops / FP32_PEAK_TFLOPS,
                        traffic=PLANE_VPSI_TRAFFIC if kname == "plane_vpsi" else None,
                        traffic_unit="DRAM bytes per launch (ncu)",
                        peak_source="FP32 CUDA-core peak from unit counts (152 SM x 128 lanes x 2 x 2.07 GHz)",
                        hbm_achieved_gbs=ach_gbs, hbm_peak_gbs=peaks.get("hbm_gbs"), hbm_peak_source=src,
                        launches=kt["launches"], avg_launch_ms=kt["ms"] / max(kt["launches"], 1),
                        share_of_step=kt["ms"] / timer_ms if timer_ms > 0 else None,
                        timed_in="a second pass of the same steps through the host-driven loop (events "
                                 "around every launch of the kernel class), after the timed region")
        line = dict(metric=METRIC, value=value, unit="evals/s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
                    ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="f32+f64" if prec == "mixed" else "f64", data="synthetic",
                    config=dict(workload=WORKLOAD, members=MEMBERS, atoms="8-32", ecut_ha=12.0, kT_ha=0.01,
                                precision=prec, start="cold (atomic density, random wavefunctions)",
                                l2="flushed by a 256 MiB write before every timed step",
                                converged=f"{n_ok}/{MEMBERS}", scf_options=dict(_SCF),
                                scf_iterations=dict(mean=float(np.mean(iters)), max=int(np.max(iters))),
                                jacobi_sweeps=dict(mean=float(np.mean(sweeps)), max=int(np.max(sweeps))),
                                eigen_refinement=dict(
                                    rule="CG steps after the SCF stopping rule until every band with "
                                         "occupation > 1e-6 has |H psi - eps psi| < 1e-4 Ha",
                                    steps_mean=float(np.mean([c["polish_steps"] for c in cstats])),
                                    steps_max=int(np.max([c["polish_steps"] for c in cstats])),
                                    max_residual=float(np.max([c["eig_resid"] for c in cstats])),
                                    jacobi_cap_hits=int(np.sum([c["jacobi_cap_hits"] for c in cstats]))),
                                autotuned=batch.tuning(), sub_batches=args.sub_batches or "auto"),
                    e2e=dict(value=e2e_val, unit="evals/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h),
                    host_loop=dict(value=ws * MEMBERS * args.steps / (timer_ms / 1e3), unit="evals/s",
                                   note="the same steps through the host-driven SCF loop with the live kernel "
                                        "timer on (sub-batches one after another); value above is the default "
                                        "graph-driven loop"),
                    gpu_launches=int(launches), roofline=roofline, clocks=clk)
        out = line
    if args.profile and rank == 0:
        prof = {}
        for kind in ("plane_vpsi", "wave_to_cols", "cols_to_wave", "plane_density", "gemm_tn", "gemm_nn", "rr",
                     "grid_fft", "cg_band", "grid_other", "gemm_small"):
            batch.timer(kind)
            a = torch.cuda.Event(enable_timing=True)
            b2 = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step_device()
            b2.record(stream)
            b2.synchronize()
            r = batch.timer_read()
            prof[kind] = dict(ms=r["ms"], launches=r["launches"], share=r["ms"] / a.elapsed_time(b2),
                              tflops=r["flops"] / max(r["ms"], 1e-9) / 1e9 if r["flops"] else None)
        batch.timer(None)
        out["profile"] = prof
    if not args.no_fp64 and rank == 0:
        # the plain FP64 GPU path on the same population, same algorithm, same stopping rule
        # and the same eigenvector refinement (FP64 arithmetic throughout, CUDA-core GEMMs,
        # FP64 eigensolve): one warm-up step, then timed steps through the same host-pointer
        # call as e2e
        ctx64 = [sgo.Context(st, precision="fp64", **_tols("mixed", st)) for st in pop]
        b64 = sgo.Batch(ctx64)
        b64.energy_forces()
        torch.cuda.synchronize()
        k64 = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        for _ in range(k64):
            E64, F64, st64 = b64.energy_forces(pos_host)
        torch.cuda.synchronize()
        dt64 = (time.perf_counter() - t0) / k64
        it64 = [c.info()["n_iter"] for c in ctx64]
        nat = np.array([c.natoms for c in ctxs])
        out["fp64_path"] = dict(value=MEMBERS / dt64, unit="evals/s", steps=k64,
                                stopping_rule="the mixed path's (|dF| < 1e-7 Ha/atom, density residual < 1e-5)",
                                converged=f"{int(np.sum(st64 == 0))}/{MEMBERS}",
                                scf_iterations=dict(mean=float(np.mean(it64)), max=int(np.max(it64))),
                                speedup_mixed_over_fp64=e2e_val / (MEMBERS / dt64),
                                max_abs_dE_per_atom_mixed_vs_fp64=float(np.max(np.abs(E - E64) / nat)),
                                max_abs_dforce_mixed_vs_fp64=float(max(np.abs(a - b).max() for a, b in zip(F, F64))))
        out["vs_fp64_gpu"] = out["fp64_path"]["speedup_mixed_over_fp64"]
        del b64, ctx64
    if not args.no_variants and rank == 0:
        out["eigensolver_variants"] = _variant_record(sgo, pop, pos_host, E, F, args)
    if rank == 0 and not args.no_warm:
        out["warm"] = _warm_steps(args, sgo, batch, ctxs, pop, pos_host, pos_dev, e_dev, f_dev, s_dev, stream)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        i = _smallest(pop)
        dt, ref = _oracle_eval(pop[i])
        out["cpu_baseline"] = dict(value=1.0 / dt, unit="evals/s", cores=_cores(), kind="oracle",
                                   sample=f"one evaluation of member {i} ({pop[i].natoms} atoms), {dt:.1f} s")
        Fi, fi = E[i], F[i]
        out["accuracy_vs_oracle"] = dict(member=i, dE_per_atom=abs(Fi - ref.free_energy) / pop[i].natoms,
                                         max_dF=float(np.max(np.abs(fi - ref.forces))))
        out["error_ledger"] = _ledger(sgo, pop[i], prec, ref, i)
    if rank == 0 and not args.no_config5:
        # the 55-atom cluster (128^3, 330 bands) one structure at a time: mixed and plain FP64
        out["config5"] = _config_record(sgo, "cluster55", stream)
    if rank == 0 and not args.no_kpoints:
        # the diamond cell on a 2 x 2 x 2 k mesh (zone folding: the 64-atom supercell at Gamma)
        out["k_points"] = _config_record(sgo, "diamond8_k222", stream, kernels=False)
    if rank == 0 and not args.no_relax:
        out["relax"] = _relax_population(sgo, batch, ctxs, pop, method=args.relax_method)
        out["de_search"] = _de_search(sgo)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _variant_record(sgo, pop, pos_host, E, F, args):
    """Variants on the same population, precision and stopping rule, each against the default
    path: the block Davidson eigensolver (2 n_b Rayleigh-Ritz over [X, W] per step) in place of
    Algorithm 1's all-band CG (same energies), PBE in place of LDA, and a p channel added to
    every species' projectors (three more projectors per atom; PBE and the p channel change the
    Hamiltonian: their energy differences are the model's).  Evals/s through the host-pointer
    call, SCF iterations, Jacobi sweeps per member."""
    import torch
    rec = {}
    nat = np.array([st.natoms for st in pop])
    import dataclasses
    import workloads
    pop_p = [dataclasses.replace(st, species=[dict(sp, **{k: workloads.SPECIES_Z4_P[k] for k in workloads.SPECIES_P_KEYS})
                                              for sp in st.species]) for st in pop]
    for name, extra, members in (("davidson", dict(eigensolver="davidson"), pop), ("pbe", dict(xc="pbe"), pop),
                                 ("p_channel", {}, pop_p)):
        ctxv = [sgo.Context(st, precision=args.precision, **extra, **_tols(args.precision, st)) for st in members]
        bv = sgo.Batch(ctxv)
        bv.energy_forces()
        torch.cuda.synchronize()
        k = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        for _ in range(k):
            Ev, Fv, sv = bv.energy_forces(pos_host)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / k
        its = [c.info()["n_iter"] for c in ctxv]
        sweeps = [c.stats()["jacobi_sweeps"] for c in ctxv]
        rec[name] = dict(value=len(pop) / dt, unit="evals/s", steps=k,
                         converged=f"{int(np.sum(sv == 0))}/{len(pop)}",
                         scf_iterations=dict(mean=float(np.mean(its)), max=int(np.max(its))),
                         jacobi_sweeps_per_member=float(np.mean(sweeps)),
                         max_abs_dE_per_atom_vs_default=float(np.max(np.abs(E - Ev) / nat)),
                         max_abs_dforce_vs_default=float(max(np.abs(a - b).max() for a, b in zip(F, Fv))))
        del bv, ctxv
    return rec


def _config_record(sgo, name, stream, kernels=True, fp64=True, extra=None):
    """One named workload on its own: for the mixed and (fp64) the plain FP64 GPU path, one
    cold energy + force evaluation timed after a warm-up evaluation (graph-driven SCF loop),
    its SCF iterations and eigenvector refinement, its errors against the stored oracle
    ledger where one exists (tests/golden/ledger_<name>.json), and (kernels) for the mixed
    path the live-timed plane pass, tensor-core GEMMs and subspace eigensolve of one more
    evaluation with their FP32-peak and tensor fractions."""
    import torch
    import workloads
    st = workloads.CONFIGS[name]()
    gold = os.path.join(ROOT, "tests", "golden", f"ledger_{name}.json")
    # (the stored ledgers are LDA results)
    ref = json.load(open(gold)) if os.path.exists(gold) and (extra or {}).get("xc", "lda") == "lda" else None
    peaks, src = _peaks()
    res = {}
    for prec in ("mixed", "fp64") if fp64 else ("mixed",):
        tol = _tols(prec, st) if name.startswith("diamond8") and prec == "fp64" else _tols("mixed", st)
        if name.startswith("diamond8"):
            tol.update(mix_alpha=0.7, kerker_q0=0.0)
        tol.update(extra or {})
        try:
            ctx = sgo.Context(st, precision=prec, **tol)
        except sgo.SgoError as e:
            res[prec] = dict(unavailable=str(e))
            continue
        b = sgo.Batch([ctx])
        b.energy_forces()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        E, F, stat = b.energy_forces()
        z.record(stream)
        z.synchronize()
        ms = a.elapsed_time(z)
        r = dict(evals_per_s=1e3 / ms, ms_per_eval=ms, status=int(stat[0]), **ctx.stats())
        eig, occ = ctx.eigen()
        if ref is not None:
            oc = np.array(ref["occ"]) > 1e-6
            if np.ndim(ref["eig"]) == 2:
                # a k mesh: the oracle holds n_b bands per k point, the folded cell the lowest
                # n_k n_b states of the mesh; both are complete below the oracle's lowest top
                # band, and the occupied states below it (less 2 mHa) are compared, sorted
                ek = np.array(ref["eig"])
                lim = min(float(ek[:, -1].min()), float(np.max(eig))) - 2e-3
                e_ref = np.sort(ek[oc & (ek < lim)])
                deig = float(np.abs(np.sort(eig)[:len(e_ref)] - e_ref).max())
            else:
                deig = float(np.abs(eig - np.array(ref["eig"]))[oc].max())
            r["errors_vs_oracle"] = dict(dF_per_atom=abs(E[0] - ref["free_energy"]) / st.natoms,
                                         max_dforce=float(np.abs(F[0] - np.array(ref["forces"])).max()),
                                         max_deig_occupied=deig)
        r["_E"], r["_F"], r["_eig"] = float(E[0]), F[0], eig
        if prec == "mixed" and kernels:
            kern = {}
            for kind in ("plane_vpsi", "gemm_tn", "gemm_nn", "rr"):
                b.timer(kind)
                a.record(stream)
                b.energy_forces()
                z.record(stream)
                z.synchronize()
                t = b.timer_read()
                tf = t["flops"] / max(t["ms"], 1e-9) / 1e9
                kern[kind] = dict(ms=t["ms"], launches=t["launches"], share=t["ms"] / a.elapsed_time(z),
                                  tflops=tf, gbs=t["bytes"] / max(t["ms"], 1e-9) / 1e6)
                if kind == "plane_vpsi":
                    kern[kind]["frac_fp32_peak"] = tf / FP32_PEAK_TFLOPS
                if kind in ("gemm_tn", "gemm_nn"):
                    if ctx.info()["nbands"] + 4 + ctx.info()["nbands"] // 32 <= 128:
                        # tcgen05 3xTF32: three tensor MMAs per useful flop, against the TF32
                        # rate (half the measured BF16 dense rate)
                        kern[kind]["units"] = "tensor cores (tcgen05, 3xTF32)"
                        kern[kind]["frac_tf32_tensor_peak"] = 3 * tf / (0.5 * peaks.get("bf16_tflops", 1900.0))
                    else:
                        kern[kind]["units"] = "CUDA cores (FP32; the tensor-core GEMMs take up to 128 bands)"
                        kern[kind]["frac_fp32_peak"] = tf / FP32_PEAK_TFLOPS
            b.timer(None)
            r["kernels"] = kern
        res[prec] = r
        del b, ctx
    if "_E" in res.get("mixed", {}) and "_E" in res.get("fp64", {}):
        m, f = res["mixed"], res["fp64"]
        res["mixed_vs_fp64"] = dict(dF_per_atom=abs(m["_E"] - f["_E"]) / st.natoms,
                                    max_dforce=float(np.abs(m["_F"] - f["_F"]).max()),
                                    max_deig=float(np.abs(m["_eig"] - f["_eig"]).max()),
                                    speedup=m["evals_per_s"] / f["evals_per_s"])
    for prec in ("mixed", "fp64"):
        for k in ("_E", "_F", "_eig"):
            res.get(prec, {}).pop(k, None)
    return dict(natoms=st.natoms, nbands=st.nbands, grid=list(st.fft), kgrid=list(st.kgrid), **res)


def run_configs(args):
    """Per-config measurement: the named workloads one structure at a time (_config_record).
    One JSON line per config, then one with all."""
    import torch
    import paper_1603_02732_gb300 as sgo
    from paper_1603_02732_gb300 import build
    build.build()
    sgo.load_library()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    names = args.names.split(",") if args.names else ["diamond8", "honeycomb24", "cluster13", "cluster55"]
    out = {}
    extra = dict(eigensolver=args.eigensolver) if args.eigensolver else {}
    if args.xc:
        extra["xc"] = args.xc
    for k, v in (("ncg", args.ncg), ("ncg_first", args.ncg_first), ("n_nonscf", args.nonscf)):
        if v is not None:
            extra[k] = v
    for name in names:
        out[name] = _config_record(sgo, name, stream, fp64=not args.no_fp64, extra=extra)
        print(json.dumps({name: out[name]}), flush=True)
    print(json.dumps(dict(case="configs", results=out)), flush=True)
    return 0


def run_case(args):
    """Small single-member cases for kernel captures: three H psi applies with a random
    potential (--case hpsi), or one SCF + forces (--case scf)."""
    import paper_1603_02732_gb300 as sgo
    from paper_1603_02732_gb300 import build
    import workloads
    build.build()
    st = workloads.de_candidate(args.member)
    extra = dict(eigensolver=args.eigensolver) if args.eigensolver else {}
    if args.xc:
        extra["xc"] = args.xc
    ctx = sgo.Context(st, precision=args.precision, **_tols(args.precision, st), **extra)
    if args.case == "hpsi":
        rng = np.random.default_rng(0)
        v = rng.normal(size=ctx.grid) * 0.1
        x = rng.normal(size=(st.nbands, ctx.npw))
        for _ in range(3):
            y = ctx.apply_hamiltonian(v, x)
        print(json.dumps(dict(case="hpsi", member=args.member, natoms=st.natoms, nbands=st.nbands,
                              grid=list(ctx.grid), npw=ctx.npw, max_abs=float(np.abs(y).max()))))
    else:
        F, _ = ctx.energy_forces()
        print(json.dumps(dict(case="scf", member=args.member, natoms=st.natoms, F=F, **ctx.stats())))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--kernel", default="plane_vpsi", help="kernel class timed live for the roofline")
    ap.add_argument("--no-fp64", action="store_true", help="skip timing the plain FP64 GPU path")
    ap.add_argument("--no-config5", action="store_true", help="skip the 55-atom cluster record")
    ap.add_argument("--no-kpoints", action="store_true", help="skip the k-mesh (diamond cell, 2x2x2) record")
    ap.add_argument("--no-variants", action="store_true", help="skip the block Davidson eigensolver record")
    ap.add_argument("--eigensolver", default=None, choices=["cg", "davidson"],
                    help="--case configs / scf: the eigensolver (default: the library's, Algorithm 1's CG)")
    ap.add_argument("--xc", default=None, choices=["lda", "pbe"],
                    help="--case configs / scf: exchange-correlation (default LDA)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven SCF loop instead of the captured graphs (for per-kernel profilers, "
                         "which cannot look inside graphs with conditional nodes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warm", action="store_true", help="skip the warm-start (relaxation step) measurement")
    ap.add_argument("--no-relax", action="store_true", help="skip the local-relaxation (PCG) measurement")
    ap.add_argument("--relax-method", default="pcg", choices=["pcg", "cg", "bfgs"])
    ap.add_argument("--sub-batches", type=int, default=0,
                    help="sub-batches overlapped on the GPU in graph mode (0 = the library's choice)")
    ap.add_argument("--profile", action="store_true", help="one extra step per kernel class with live timers")
    ap.add_argument("--case", default="batch", choices=["batch", "hpsi", "scf", "configs"],
                    help="batch: the benchmark; hpsi / scf: one population member (small case for ncu); "
                         "configs: the named workloads one at a time (mixed and FP64)")
    ap.add_argument("--names", default=None, help="--case configs: comma-separated workload names")
    ap.add_argument("--member", type=int, default=0, help="population member for --case hpsi / scf")
    ap.add_argument("--ncg", type=int, default=None, help="CG steps per SCF iteration")
    ap.add_argument("--ncg-first", type=int, default=None)
    ap.add_argument("--nonscf", type=int, default=None)
    ap.add_argument("--extra-bands", type=int, default=None, help="headroom bands (default: the library's)")
    ap.add_argument("--rr-cluster", type=int, default=None, choices=[0, 1],
                    help="subspace eigensolve on an 8-CTA cluster per member (1) or one CTA (0)")
    ap.add_argument("--cg-adapt", type=float, default=None,
                    help="density residual above which an SCF iteration takes one CG step fewer")
    ap.add_argument("--mix-alpha", type=float, default=None, help="Pulay step (default: the library's)")
    ap.add_argument("--pulay-hist", type=int, default=None, help="Pulay history (default: the library's)")
    ap.add_argument("--kerker-q0", type=float, default=None, help="Kerker q0 (default: the library's)")
    args = ap.parse_args()
    for k, v in (("ncg", args.ncg), ("ncg_first", args.ncg_first), ("n_nonscf", args.nonscf),
                 ("extra_bands", args.extra_bands), ("mix_alpha", args.mix_alpha), ("pulay_hist", args.pulay_hist),
                 ("cg_adapt", args.cg_adapt), ("rr_cluster", args.rr_cluster), ("kerker_q0", args.kerker_q0)):
        if v is not None:
            _SCF[k] = v
    if args.no_graph:
        _SCF["graph"] = 0
    if args.impl == "reference":
        return run_reference(args)
    if args.case == "configs":
        return run_configs(args)
    if args.case != "batch":
        return run_case(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
