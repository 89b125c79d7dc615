#!/usr/bin/env python
"""Benchmark of the FEF effective-field Fock build and FEF self-consistency on GB300.

Workload: 64 water-like fragments (O 3s2p, H 2s, 3 primitives per shell, seeded random bases) in a
12.42 A cube at 1 g/cm^3, 8 A fragment-pair cutoff, Schwarz 1e-12, FEF converged to 1e-8 Eh.

One step = one complete pass of the hot path on one synthetic snapshot through the public C ABI:
fef_create (normalisation, Boys table, one-electron and intra-fragment integrals, neighbour list,
nuclear field, orthogonalisers, work lists) + fef_iterate (superposition start, macro-iterations of
Hermite densities, J-engine, Fock assembly, device fragment SCF, energies) + fef_energies.

value  = inter-fragment shell quartets processed (surviving quartets x Fock builds) / device time,
         CUDA events on the context stream, L2 flushed (256 MiB write) between steps; FP64 mode,
         native FP64 J-engine.
Legs reported beside it (same workload, same 1e-8 Eh convergence, energies compared to FP64):
  df64                 FP64-accurate solve with the float-float J-engine (FP32 pipes);
  mixed_fp64_reference MIXED: FP32-core increments, native FP64 reference build;
  mixed                MIXED with the float-float reference build;
  mixed_learned        MIXED (float-float reference) from the learned warm start; the network is
                       trained beforehand (not timed) on 40 seeded snapshots drawn like the workload.
learned_2000_waters: the learned start at full size, reduced: trained on 8 x 500-water boxes (not
       timed), MIXED solves of 2 held-out 2000-water boxes from the superposition and the learned start.
e_m2 / e_d2: one fef_energy_m2 / fef_energy_d2 call on the converged FP64 state (second-order
       energies, Eqs. EM2 and ED2), wall clock.
heterocycle_1000_waters: the precision workload, a 130-AO C4N3OH5-like solute with s/p/d shells in
       1000 waters (31 A cube, 8 A cutoff): the FP32 core's own error (one whole-density build of the
       isolated densities against the FP64 build, per fragment and per Fock element), and the time
       to 1e-8 Eh of FP64 and of MIXED (float-float reference) solves with autotuned tile plans.
e2e    = the same step plus the device->host read of every converged density, wall clock.
roofline: the J-engine (one persistent FP64 launch per Fock build) against the FP64 ALU peak.
--impl reference: the CPU oracle on a bounded sample of the same workload.

Multi-GPU (torchrun): independent replicas, one snapshot per rank (seed = rank), no collective
on the data path; value sums all ranks' quartets over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FEF shell quartets/s & time to 1e-8 Eh FEF: mixed+learned vs FP64 (1 GB300)"
UNIT = "shell quartets/s"
WORKLOAD = "64 water-like fragments, 12.42 A cube (1 g/cm^3), 8 A cutoff, Schwarz 1e-12, FEF to 1e-8 Eh, FP64"
N_WATER, CUTOFF_A, SCHWARZ, E_TOL = 64, 8.0, 1e-12, 1e-8
SMS, SM_MAX_MHZ = 152, 2070.0
# GB300 FP64: 1.25 TFLOP/s nominal = 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz
FP64_PEAK = SMS * 2 * 2 * SM_MAX_MHZ * 1e6


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------------------------------- flop model
def nh(L):
    return (L + 1) * (L + 2) * (L + 3) // 6


def flops_per_prim_quartet(LP, LQ):
    """Algorithmic FP64 work of one primitive quartet of Hermite class (L_P, L_Q) in the fused
    J-engine: 40 (setup, Boys, prefactor) + 3 per R^{(n)}_{tuv} of the MD recursion + 2 N(L_P) N(L_Q)
    for the two contractions (field on the bra and on the ket)."""
    L = LP + LQ
    return 40 + 3 * sum(nh(k) for k in range(L + 1)) + 2 * nh(LP) * nh(LQ)


def algorithmic_flops(class_quartets):
    cq = np.asarray(class_quartets).reshape(5, 5)
    return float(sum(cq[a, b] * flops_per_prim_quartet(a, b) for a in range(5) for b in range(5)))


# ----------------------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        out_dir = os.environ.get("FEF_BENCH_OUT", os.path.join(tempfile.gettempdir(), "fef_bench"))
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------------------- helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def profile_traffic():
    """DRAM bytes per J-engine build from the committed ncu summary, if it was taken on the
    current J-engine sources (jengine.cu and common.cuh, matching hashes); else None."""
    path = os.path.join(ROOT, "profiles", "jengine_water64_fp64.txt")
    csrc = os.path.join(ROOT, "paper_1708_03377_gb300", "csrc")
    if not os.path.exists(path):
        return None
    want = {k: hashlib.sha1(open(os.path.join(csrc, f), "rb").read()).hexdigest()[:12]
            for k, f in (("jengine_source_sha1", "jengine.cu"), ("common_source_sha1", "common.cuh"))}
    got, traffic = {}, None
    for line in open(path):
        key = line.split(":", 1)[0]
        if key in want:
            got[key] = line.split(":", 1)[1].strip()
        if key == "dram_bytes_per_build":
            traffic = float(line.split(":", 1)[1].strip())
    return traffic if got == want else None


def cpu_baseline(seconds=12.0):
    """The CPU oracle on a bounded sample of the workload: Obara-Saika ERI blocks and the J
    contraction for the first fragment pairs of the neighbour list (shell quartets/s)."""
    from oracle import integrals as I
    from synth import systems as S
    system = S.water_box(N_WATER, seed=0)
    nf = system.n_frag
    shells = [I.fragment_shells(system, x) for x in range(nf)]
    t0 = time.perf_counter()
    Q = [s.schwarz() for s in shells]
    pairs = []
    xyz = system.xyz
    for x in range(nf):
        ax = system.frag_atoms(x)
        for y in range(x + 1, nf):
            ay = system.frag_atoms(y)
            if np.linalg.norm(xyz[ax][:, None] - xyz[ay][None], axis=-1).min() < CUTOFF_A:
                pairs.append((x, y))
    rng = np.random.default_rng(0)
    quartets, done = 0, 0
    for x, y in pairs:
        e = I.eri_block(shells[x], shells[y], Q[x], Q[y], SCHWARZ)
        nx, ny = shells[x].n_ao, shells[y].n_ao
        D = rng.standard_normal((ny, ny))
        _ = e.reshape(nx * nx, ny * ny) @ (D + D.T).ravel()
        quartets += I.count_quartets(shells[x], shells[y], Q[x], Q[y], SCHWARZ)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": quartets / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"Schwarz factors of all 64 fragments + Obara-Saika ERI blocks and J contraction of the "
                      f"first {done} of {len(pairs)} fragment pairs ({quartets} shell quartets, {dt:.1f} s)"}


def oracle_time_to_converge():
    """The oracle's own FEF solve of the whole workload to 1e-8 Eh (integrals, superposition start,
    macro-iterations), wall clock on the host cores: the time-to-convergence the GPU legs are compared with."""
    from oracle.fef import Fragments
    from synth import systems as S
    t0 = time.perf_counter()
    fr = Fragments(S.water_box(N_WATER, seed=0), cutoff_A=CUTOFF_A, schwarz=SCHWARZ)
    t1 = time.perf_counter()
    res = fr.solve(e_tol=E_TOL)
    t2 = time.perf_counter()
    return {"time_to_1e-8_s": t2 - t0, "integrals_s": t1 - t0, "n_macro": res["n_macro"],
            "E_tot": res["energies"]["E_tot"],
            "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}


# ----------------------------------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    vals, times = [], []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(seconds=args.ref_seconds)
        if i >= args.warmup:
            vals.append(r["value"])
            times.append(float(r["sample"].split(", ")[-1].split(" s")[0]))
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (bounded sample per step)", "n_frag": N_WATER,
                       "cutoff_A": CUTOFF_A, "schwarz": SCHWARZ},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------- our arm
def reduce_over_replicas(dist, total_ms, quartets, launches, device):
    """Whole-job figures of independent replicas: the slowest rank's time, the summed shell quartets
    and kernel launches of all ranks (one collective pair, outside the timed region)."""
    import torch
    t = torch.tensor([total_ms, float(quartets), float(launches)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1]), int(t[2])


def heterocycle_leg(fef, S, stream):
    """The precision workload: FP32-core whole build vs FP64 build of the isolated densities (per
    fragment energy and Fock element errors), and FP64 vs MIXED time to 1e-8 Eh (CUDA events around
    fef_iterate, after the isolated RHF and autotuning of the engines used)."""
    import torch
    system = S.solvated_heterocycle(n_water=1000, seed=0)
    cut = 8.0

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1)

    with torch.cuda.stream(stream):
        o64 = fef.fef_default_options(cutoff_A=cut, schwarz=SCHWARZ, e_tol=E_TOL, use_graph=0)
        t0 = time.perf_counter()
        ctx = fef.fef_create_system(system, o64, stream=stream.cuda_stream)
        stream.synchronize()
        create_s = time.perf_counter() - t0
        fef.fef_noninteracting_scf(ctx)
        Diso = fef.fef_get_densities(ctx)
        fef.fef_build_fock(ctx, Diso)
        F64, b64_ms = timed(lambda: fef.fef_build_fock(ctx, Diso))
        E64, _, _ = fef.fef_energies(ctx)
        n0 = int(ctx.n_ao[0])  # the solute is fragment 0
        ctx.close()
        ow = fef.fef_default_options(cutoff_A=cut, schwarz=SCHWARZ, e_tol=E_TOL, precision=fef.FEF_MIXED,
                                     mixed_build=fef.FEF_MIXED_WHOLE, use_graph=0)
        ctx = fef.fef_create_system(system, ow, stream=stream.cuda_stream)
        fef.fef_build_fock(ctx, Diso)
        F32, b32_ms = timed(lambda: fef.fef_build_fock(ctx, Diso))
        E32, _, _ = fef.fef_energies(ctx)
        ctx.close()
        dE = E32 - E64
        dF = np.abs(F32 - F64)
        solves = {}
        for name, opts, engines in (
                ("fp64", fef.fef_default_options(cutoff_A=cut, schwarz=SCHWARZ, e_tol=E_TOL), [fef.FEF_JENGINE_FP64]),
                ("mixed", fef.fef_default_options(cutoff_A=cut, schwarz=SCHWARZ, e_tol=E_TOL, precision=fef.FEF_MIXED,
                                                  exact_engine=fef.FEF_ENGINE_DF64),
                 [fef.FEF_JENGINE_DF64, fef.FEF_JENGINE_FP32])):
            ctx = fef.fef_create_system(system, opts, stream=stream.cuda_stream)
            fef.fef_noninteracting_scf(ctx)
            for e in engines:
                fef.fef_autotune(ctx, e, reps=2, budget_ms=4000.0)
            (n_macro, _), it_ms = timed(lambda: fef.fef_iterate(ctx))
            _, E_tot, _ = fef.fef_energies(ctx)
            E_x = fef.fef_energies(ctx)[0]
            solves[name] = {"time_to_1e-8_ms": it_ms, "n_macro": int(n_macro), "E_tot": float(E_tot), "E_x": E_x}
            ctx.close()
    dEs = solves["mixed"]["E_x"] - solves["fp64"]["E_x"]
    for v in solves.values():
        del v["E_x"]
    return {"workload": system.name + ", 8 A cutoff, Schwarz 1e-12", "n_frag": int(system.n_frag),
            "solute_nao": int(n0), "create_s": create_s,
            "fp32_whole_build": {"max_dE_x": float(np.abs(dE).max()), "rms_dE_x": float(np.sqrt(np.mean(dE ** 2))),
                                 "solute_dE": float(dE[0]), "max_dF": float(dF.max()),
                                 "solute_max_dF": float(dF[:n0 * n0].max()),
                                 "fp32_build_ms": b32_ms, "fp64_build_ms": b64_ms,
                                 "note": "FP32-core J-engine of the whole isolated density (no FP64 reference) "
                                         "against the FP64 build (hartree)"},
            "fp64": solves["fp64"], "mixed": solves["mixed"],
            "mixed_speedup_vs_fp64": solves["fp64"]["time_to_1e-8_ms"] / solves["mixed"]["time_to_1e-8_ms"],
            "mixed_converged": {"max_dE_x_vs_fp64": float(np.abs(dEs).max()),
                                "dE_tot_vs_fp64": solves["mixed"]["E_tot"] - solves["fp64"]["E_tot"]}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=8.0)
    ap.add_argument("--no-learned-2000", action="store_true",
                    help="skip the reduced full-size learned-start leg (2000-water held-out boxes)")
    ap.add_argument("--no-heterocycle", action="store_true",
                    help="skip the precision leg (130-AO solute in 1000 waters)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import paper_1708_03377_gb300 as fef
    from synth import systems as S

    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    stream = torch.cuda.Stream()
    system = S.water_box(N_WATER, seed=rank)
    # FP64 leg with eager launches: its J-engine time per build comes from CUDA events on the
    # context stream (inside a captured graph the library times phases with device timestamps)
    opts = fef.fef_default_options(cutoff_A=CUTOFF_A, schwarz=SCHWARZ, e_tol=E_TOL, use_graph=0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fef.lib()
    fp64_probe, fp32_probe, _ = fef.fef_measure_fma_peak()

    def one_step(read_back=False, options=None, warm=None):
        ctx = fef.fef_create_system(system, options or opts, stream=stream.cuda_stream)
        if warm is not None:
            fef.fef_set_warm_start(ctx, warm)
        t_it0 = torch.cuda.Event(enable_timing=True)
        t_it1 = torch.cuda.Event(enable_timing=True)
        t_it0.record(stream)
        n_macro, dE = fef.fef_iterate(ctx)
        t_it1.record(stream)
        E_frag, E_tot, _ = fef.fef_energies(ctx)
        D = fef.fef_get_densities(ctx) if read_back else None
        st = fef.fef_stats(ctx)
        hist = fef.fef_history(ctx)
        ctx.close()
        return dict(n_macro=n_macro, E_tot=E_tot, stats=st, ev=(t_it0, t_it1), D=D, hist=hist)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        launches0 = fef.fef_stats()["kernel_launches"]
        step_ms, iter_ms, quartets, results = [], [], 0, []
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            if pg:
                pg.barrier()
            wall0 = time.perf_counter()
            for k in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = one_step()
                e1.record(stream)
                e1.synchronize()
                step_ms.append(e0.elapsed_time(e1))
                iter_ms.append(r["ev"][0].elapsed_time(r["ev"][1]))
                quartets += r["stats"]["shell_quartets"] * (r["n_macro"] + 1)
                results.append(r)
            torch.cuda.synchronize()
            if pg:
                pg.barrier()
            wall = time.perf_counter() - wall0
        launches = fef.fef_stats()["kernel_launches"] - launches0
        clocks = clk.summary()
        # MIXED: FP32-core incremental builds + FP64 reference refresh (same workload, to 1e-8 Eh)
        def variant(options, warm=None):
            it_ms, step_ms, res = [], [], None
            for k in range(args.warmup + max(2, args.steps // 2)):
                flush.zero_()
                m0 = torch.cuda.Event(enable_timing=True)
                m1 = torch.cuda.Event(enable_timing=True)
                m0.record(stream)
                res = one_step(options=options, warm=warm)
                m1.record(stream)
                m1.synchronize()
                if k >= args.warmup:
                    it_ms.append(res["ev"][0].elapsed_time(res["ev"][1]))
                    step_ms.append(m0.elapsed_time(m1))
            return it_ms, step_ms, res

        def summary(it_ms, step_ms, res):
            return {"time_to_1e-8_ms": float(np.mean(it_ms)), "ms_per_step": float(np.mean(step_ms)),
                    "n_macro": res["n_macro"],
                    "fp32_builds": int(sum(h["fp32"] for h in res["hist"])),
                    "fp64_builds": int(sum(1 - h["fp32"] for h in res["hist"])),
                    "E_tot_minus_fp64": res["E_tot"] - results[-1]["E_tot"],
                    "value": res["stats"]["shell_quartets"] * (res["n_macro"] + 1) / (float(np.mean(step_ms)) * 1e-3),
                    "speedup_time_to_1e-8_vs_fp64": float(np.mean(iter_ms)) / float(np.mean(it_ms))}

        DF = fef.FEF_ENGINE_DF64
        # FP64-accurate solve with the float-float J-engine (same iteration, FP64 eigensolve/energies)
        dopts = fef.fef_default_options(cutoff_A=CUTOFF_A, schwarz=SCHWARZ, e_tol=E_TOL, exact_engine=DF)
        df_ms, df_step_ms, dres = variant(dopts)
        # MIXED with the native FP64 reference build, and with the float-float one
        mfopts = fef.fef_default_options(cutoff_A=CUTOFF_A, schwarz=SCHWARZ, e_tol=E_TOL, precision=fef.FEF_MIXED)
        mixed64_ms, mixed64_step_ms, m64res = variant(mfopts)
        mopts = fef.fef_default_options(cutoff_A=CUTOFF_A, schwarz=SCHWARZ, e_tol=E_TOL, precision=fef.FEF_MIXED,
                                        exact_engine=DF)
        mixed_ms, mixed_step_ms, mres = variant(mopts)
        # the FP32 core on its own (no FP64 reference): one whole-density build of the isolated densities
        # against the FP64 build of the same densities, per-fragment energies and Fock elements (not timed)
        wctx = fef.fef_create_system(system, opts, stream=stream.cuda_stream)
        fef.fef_noninteracting_scf(wctx)
        Diso = fef.fef_get_densities(wctx)
        F64w = fef.fef_build_fock(wctx, Diso)
        E64w, _, _ = fef.fef_energies(wctx)
        wctx.close()
        wopts = fef.fef_default_options(cutoff_A=CUTOFF_A, schwarz=SCHWARZ, e_tol=E_TOL, precision=fef.FEF_MIXED,
                                        mixed_build=fef.FEF_MIXED_WHOLE, use_graph=0)
        wctx = fef.fef_create_system(system, wopts, stream=stream.cuda_stream)
        F32w = fef.fef_build_fock(wctx, Diso)
        E32w, _, _ = fef.fef_energies(wctx)
        wctx.close()
        dEw = E32w - E64w
        fp32_whole = {"max_dE_x": float(np.abs(dEw).max()), "rms_dE_x": float(np.sqrt(np.mean(dEw ** 2))),
                      "mean_dE_x": float(dEw.mean()), "max_dF": float(np.abs(F32w - F64w).max()),
                      "note": "FP32-core J-engine of the whole isolated density (no FP64 reference) against the "
                              "FP64 build, per fragment (hartree)"}
        # E_M2 (Eq. EM2) on the converged FP64 state: one public call (intra-fragment integrals
        # recomputed, canonical orbitals, four quarter-transforms, second-order sum), wall clock
        m2ctx = fef.fef_create_system(system, opts, stream=stream.cuda_stream)
        fef.fef_iterate(m2ctx)
        m2_ms, m2_tot, d2_ms, d2_tot = [], 0.0, [], 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, m2_tot = fef.fef_energy_m2(m2ctx)
            m2_ms.append(1e3 * (time.perf_counter() - t0))
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, d2_tot = fef.fef_energy_d2(m2ctx)
            d2_ms.append(1e3 * (time.perf_counter() - t0))
        m2ctx.close()
        nao_w = S.frag_n_ao(system, 0)
        nocc_w = S.frag_n_occ(system, 0)
        nv_w, np_w = nao_w - nocc_w, nao_w * (nao_w + 1) // 2
        m2_flop = 2.0 * N_WATER * (nocc_w * nao_w * np_w * nao_w + nocc_w * nv_w * np_w * nao_w
                                   + nocc_w * nv_w * nocc_w * nao_w * nao_w + (nocc_w * nv_w) ** 2 * nao_w)
        # MIXED + learned warm start: the network is trained beforehand (not timed) on converged densities
        # of 40 seeded snapshots drawn like the workload (64 waters at 1 g/cm^3, its basis)
        from paper_1708_03377_gb300 import learned as lrn
        Xs, Ts = [], []
        for sd in range(1000, 1040):
            try:
                Xq, Tq = lrn.snapshot_samples(S.water_box(N_WATER, seed=sd, basis_sets=system.basis_sets),
                                              cutoff_A=CUTOFF_A)
                Xs.append(Xq)
                Ts.append(Tq)
            except fef.FefError:
                pass
        net, net_loss = lrn.train_warm_start(np.concatenate(Xs), np.concatenate(Ts), hidden=256, epochs=300, batch=128)
        lopts = fef.fef_default_options(cutoff_A=CUTOFF_A, schwarz=SCHWARZ, e_tol=E_TOL, precision=fef.FEF_MIXED,
                                        start=fef.FEF_START_LEARNED, exact_engine=DF)
        ml_ms, ml_step_ms, mlres = variant(lopts, warm=net)
        # e2e: the same step through the public API plus the density read-back, wall clock
        e2e_ms = []
        for k in range(max(2, args.steps // 2)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = one_step(read_back=True)
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
        torch.cuda.synchronize()

    # learned start at full size, reduced: trained on 8 x 500 waters (every fragment, not timed),
    # then MIXED from the superposition and from the learned start on 2 held-out 2000-water boxes
    # (time to 1e-8 Eh of fef_iterate by CUDA events, after one untimed solve per leg)
    learned_2000 = None
    if not args.no_learned_2000 and rank == 0:
        learned_2000 = lrn.run_experiment(train_snapshots=8, train_waters=500, per_snapshot=500, test_snapshots=2,
                                          test_waters=2000, fp64_test_snapshots=0, cutoff=CUTOFF_A, e_tol=E_TOL,
                                          epochs=200, warmup=1)
    hetero = None
    if not args.no_heterocycle and rank == 0:
        hetero = heterocycle_leg(fef, S, stream)
    total_ms = float(sum(step_ms))
    if pg:
        total_ms, quartets, launches = reduce_over_replicas(pg, total_ms, quartets, launches, "cuda")
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    last = results[-1]
    st = last["stats"]
    builds = last["n_macro"] + 1
    jms_per_build = float(np.mean([h["jengine_ms"] for h in last["hist"]]))  # every build of the FP64 solve
    flops_build = algorithmic_flops(st["class_quartets"])
    achieved = flops_build / (jms_per_build * 1e-3)
    jms32 = float(np.mean([h["jengine_ms"] for h in mres["hist"] if h["fp32"]] or [float("nan")]))
    value = quartets / (total_ms * 1e-3)
    so, sl, sn, ex, co = system.flat_basis()
    h2d = sum(a.nbytes for a in (system.Z, system.xyz, system.frag_of_atom, system.basis_of_atom, system.charge,
                                  so, sl, sn, ex, co))
    d2h = int(r["D"].nbytes) + 8 * (2 * N_WATER + 1)   # densities + E_frag, E_int, E_total
    e2e_value = st["shell_quartets"] * builds / (float(np.mean(e2e_ms)) * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_frag": N_WATER, "cutoff_A": CUTOFF_A, "schwarz": SCHWARZ,
                   "e_tol": E_TOL, "precision": "fp64", "start": "superposition", "seed": "rank",
                   "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{ws}"},
        "time_to_1e-8_ms": float(np.mean(iter_ms)), "setup_and_energies_ms": total_ms / args.steps - float(np.mean(iter_ms)),
        "n_macro": last["n_macro"], "fock_builds_per_step": builds,
        "shell_quartets_per_build": st["shell_quartets"], "prim_quartets_per_build": int(np.sum(st["class_quartets"])),
        "prim_quartets_per_s": value * float(np.sum(st["class_quartets"])) / max(st["shell_quartets"], 1),
        "jengine_shell_quartets_per_s": st["shell_quartets"] / (jms_per_build * 1e-3),
        "E_tot": last["E_tot"],
        "df64": {**summary(df_ms, df_step_ms, dres), "exact_engine": "df64 (float-float on the FP32 pipes)",
                 "jengine_ms_per_build": float(np.mean([h["jengine_ms"] for h in dres["hist"]])),
                 "fp64_equivalent_tflops": flops_build / (float(np.mean([h["jengine_ms"] for h in dres["hist"]])) * 1e-3) / 1e12},
        "mixed_fp64_reference": {**summary(mixed64_ms, mixed64_step_ms, m64res), "exact_engine": "fp64"},
        "mixed": {**summary(mixed_ms, mixed_step_ms, mres), "exact_engine": "df64",
                  "jengine_fp32_ms_per_build": jms32,
                  "fp32_whole_build": fp32_whole,
                  "roofline_fp32": {"bound": "alu", "achieved": flops_build / (jms32 * 1e-3) / 1e12,
                                    "peak": fp32_probe / 1e12, "unit": "TFLOP/s",
                                    "frac": flops_build / (jms32 * 1e-3) / fp32_probe,
                                    "peak_source": "measured: FP32 FMA-chain probe (fef_measure_fma_peak) in this run",
                                    "kernel": "k_jengine32<LP,LQ> (FP32-core class kernels on three streams)"}},
        "mixed_learned": {**summary(ml_ms, ml_step_ms, mlres), "exact_engine": "df64",
                          "train_samples": int(sum(len(x) for x in Xs)),
                          "train_loss": net_loss},
        "learned_2000_waters": learned_2000,
        "heterocycle_1000_waters": hetero,
        "e_m2": {"ms_per_call": float(min(m2_ms[1:])), "E_m2_total": m2_tot, "transform_flop": m2_flop,
                 "note": "monomer second-order energy (Eq. EM2) of all fragments on the FEF canonical orbitals"},
        "e_d2": {"ms_per_call": float(min(d2_ms[1:])), "E_d2_total": d2_tot,
                 "note": "dimer second-order energy (Eq. ED2) over the fragment pairs within the cutoff"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": FP64_PEAK / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK, "traffic": profile_traffic(),
                     "kernel": "k_jengine_persistent<0,false> (one persistent launch per Fock build: all "
                               "fragment pairs and s/p quartet classes, cost-sorted work queue)",
                     "jengine_ms_per_build": jms_per_build, "algorithmic_flop_per_build": flops_build,
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2070 MHz (1.25 TFLOP/s nominal)",
                     "fma_probe_fp64_tflops": fp64_probe / 1e12, "fma_probe_fp32_tflops": fp32_probe / 1e12},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": float(np.mean(e2e_ms))},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "wall_s": wall,
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline"]["oracle_fef_solve"] = oracle_time_to_converge()
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
