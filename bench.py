"""Benchmark of the ensemble lattice-Boltzmann UQ hot path on GB300.

One step = one whole pass of the hot path over the 4-D Taylor-Green workload (625 tensor
Gauss-Legendre samples, 256 x 256, 2000 steps, FP32 populations, FP64 statistics): equilibrium
init, the fused collide-stream-QoI time loop, final fields, gPC projection onto the 70-term
total-degree-4 Legendre basis and the mean/variance fields.  Metric: ensemble MLUPS (sum over
samples of nodes x steps per second).  The lattice arena (1.47 GB) is larger than L2 (129 MB),
so every time step streams from HBM without an explicit flush.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded slice of the same
workload (all samples, fewer time steps) and reports the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ensemble MLUPS (tgv256_gpc4d: 625 samples x 256^2 x 2000 steps, FP32 storage, FP64 gPC statistics)"
UNIT = "MLUPS"
BYTES_PER_UPDATE = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36, "fx16": 36}
# per scheme: the step kernel, its ncu name, and the version of its code; the DRAM traffic per launch
# comes from profiles/traffic_<name>_<storage>_tgv256.txt (written by --write-traffic from an ncu
# capture), used only when that file names the same version (else traffic is null)
STEP_KERNELS = {1: ("step_kernel (one-step: fused AA collide-stream-QoI, in place)", "step_kernel", "aa-npt-nbr-pair"),
                3: ("step2_kernel (two-step tiles: tile + halo collided into shared memory, streamed and "
                    "collided again, pushed to the other lattice)", "step2_kernel", "two-step-v2-packed"),
                4: ("strip2_kernel (two-step row strips: each row collided into a shared-memory ring, streamed "
                    "and collided again, pushed to the other lattice)", "strip2_kernel", "two-step-strips-v2-staged"),
                6: ("strip3w_kernel (three-step row strips at a compile-time width: each row collided into a "
                    "first shared-memory ring, streamed and collided into a second, streamed and collided again, "
                    "pushed to the other lattice)", "strip3w_kernel", "three-step-strips-fixed-width-v3")}
STEPS_PER_LAUNCH = {1: 1, 3: 2, 4: 2, 6: 3, 7: 1}


def _traffic_file(kernel: str, storage: str) -> str:
    return os.path.join(ROOT, "profiles", f"traffic_{kernel}_{storage}_tgv256.txt")


def read_traffic(kernel: str, storage: str, version: str):
    """DRAM bytes per launch of `kernel` at the bench's full size from its machine-written file."""
    try:
        with open(_traffic_file(kernel, storage)) as fh:
            kv = dict(ln.split(None, 1) for ln in fh.read().splitlines() if ln.strip() and not ln.startswith("#"))
    except OSError:
        return None
    if kv.get("kernel_version", "").strip() != version:
        return None
    return int(float(kv["traffic_bytes_per_launch_full_size"]))


def write_traffic(csv_path: str, kernel: str, storage: str, version: str, samples: int, command: str) -> str:
    """Parse an ncu CSV (--metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
    --csv --print-units base) and write the per-launch traffic of `kernel`, scaled from the captured
    sample count to the bench's 625 samples (every sample has the same size, so the traffic of a
    launch is proportional to the samples it carries)."""
    import csv

    rows = list(csv.DictReader(ln for ln in open(csv_path) if ln.startswith('"')))
    per = {}
    for r in rows:
        if kernel not in r.get("Kernel Name", ""):
            continue
        key = r.get("ID") or r.get("Id") or r.get("Kernel Name")
        unit = r.get("Metric Unit", "byte")
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1, "usecond": 1e3, "msecond": 1e6}.get(
            unit, 1)
        per.setdefault(key, {})[r["Metric Name"]] = float(r["Metric Value"].replace(",", "")) * scale
    launches = [v for v in per.values() if "dram__bytes_read.sum" in v and "dram__bytes_write.sum" in v]
    if not launches:
        raise SystemExit(f"no {kernel} launch with DRAM counters in {csv_path}")
    rd = sum(v["dram__bytes_read.sum"] for v in launches) / len(launches)
    wr = sum(v["dram__bytes_write.sum"] for v in launches) / len(launches)
    full = (rd + wr) * 625 / samples
    path = _traffic_file(kernel, storage)
    with open(path, "w") as fh:
        fh.write(f"# DRAM traffic of {kernel} per launch (ncu), written by bench.py --write-traffic\n"
                 f"# command: {command}\n"
                 f"kernel {kernel}\nkernel_version {version}\nstorage {storage}\nlaunches_captured {len(launches)}\n"
                 f"samples_captured {samples}\ndram_bytes_read_per_launch {rd:.0f}\n"
                 f"dram_bytes_write_per_launch {wr:.0f}\nscale_to_625_samples {625 / samples:.6f}\n"
                 f"traffic_bytes_per_launch_full_size {full:.0f}\n")
    return path


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _updates(samples) -> int:
    return sum(int(s.nx) * int(s.ny) * int(s.steps) for s in samples)


def run_oracle_slice(w, steps_per_sample: int, threads: int = 0):
    """Oracle on all samples of the workload for a few time steps (bounded CPU work)."""
    from oracle import lbm as olbm
    from oracle import uq as ouq

    if w.method == "gpc":
        z, _, _ = ouq.tensor_grid([w.pts_per_dim] * len(w.bounds), w.bounds)
    else:
        z, _ = ouq.mc_samples(w.n_mc, w.bounds, w.seed)
    cases = []
    for row in z:
        p = dict(zip(w.params, row))
        u0 = p.get("u0", w.base.u0)
        cases.append(olbm.Case(w.base.kind, w.base.nx, w.base.ny, steps_per_sample, p.get("nu", w.base.nu), u0,
                               amp2=p.get("zeta2", 0.0) * u0, amp3=p.get("zeta3", 0.0) * u0, u_ref=w.base.u_ref))
    t0 = time.perf_counter()
    olbm.run(cases, threads=threads)
    el = time.perf_counter() - t0
    upd = len(cases) * w.base.nx * w.base.ny * steps_per_sample
    return upd / el / 1e6, el, upd, olbm.num_threads() if threads <= 0 else threads


def bench_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import lbm as olbm
    from paper_2508_13867_gb300 import workloads as W

    olbm.build()
    w = W.tgv256_gpc4d()
    slice_steps = args.ref_slice
    for _ in range(args.warmup):
        run_oracle_slice(w, slice_steps)
    times, upd = [], 0
    for _ in range(args.steps):
        mlups, el, u, cores = run_oracle_slice(w, slice_steps)
        times.append(el)
        upd = u
    total = sum(times)
    value = upd * len(times) / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "tgv256_gpc4d", "samples": 625, "lattice": [256, 256], "time_steps": 2000,
                       "storage": "f64 (CPU oracle)", "l2": "arena larger than L2 (no flush needed)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"all 625 samples, {slice_steps} of 2000 time steps per bench step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def bench_kernel_only(args):
    """Small case for profiler captures: the first --samples samples of the 4-D workload for
    --time-steps steps, ensemble run only (no projection, no baselines)."""
    import torch

    from paper_2508_13867_gb300 import build as lib_build

    lib_build.build()
    from paper_2508_13867_gb300 import uqlb as U
    from paper_2508_13867_gb300 import workloads as W
    from paper_2508_13867_gb300.ensemble import Ensemble

    from paper_2508_13867_gb300.ensemble import sample_struct

    ens = Ensemble(0)
    if args.kernel_case == "cylinder":
        # channel samples of the cylinder workload at nd nodes per diameter (inflow +-10 %), no steady test
        smp = [sample_struct(W.channel(args.nd, u_mean=0.04 * (0.9 + 0.2 * k / max(args.samples - 1, 1)),
                                       steps=args.time_steps, steady_tol=0.0)) for k in range(args.samples)]
    else:
        w = W.tgv256_gpc4d(storage=args.storage)
        ens.setup(w)
        smp = ens.ensemble_samples(w)[: args.samples]
        for s in smp:
            s.steps = args.time_steps
            if args.lattice > 0:
                s.nx = s.ny = args.lattice
    out = {}
    strip = tuple(int(v) for v in args.strip.split(","))
    tuned = None
    if args.kernel_autotune:
        tuned = ens.autotune(smp, storage=args.storage, trial_steps=args.tune_steps, scheme=args.scheme)
    for _ in range(args.warmup + args.steps):
        ens.run_batch(smp, storage=args.storage, fields_dtype="f32", out=out, tile_rows=args.tile_rows,
                      nodes_per_thread=args.npt, rounding=args.rounding, mode=args.mode, scheme=args.scheme,
                      strip=strip)
    torch.cuda.synchronize()
    ms, st, la = U.uqlb_last_loop_time(ens.ctx)
    scheme, g_rows, g_npt = U.uqlb_last_run_geometry(ens.ctx)
    per_launch = STEPS_PER_LAUNCH.get(scheme, 1)
    nodes = sum(s.nx * s.ny for s in smp)
    gbs = BYTES_PER_UPDATE[args.storage] * nodes / (ms / max(st / per_launch, 1) / 1e3) / 1e9
    print(json.dumps({"kernel_only": True, "mode": args.mode, "scheme": scheme, "tile": [g_rows, g_npt],
                      "samples": len(smp), "time_steps": st, "mlups": nodes * st / (ms / 1e3) / 1e6,
                      "storage": args.storage,
                      "loop_ms": ms, "step_ms": ms / max(st, 1), "achieved_gbs": gbs,
                      "arena_bytes": BYTES_PER_UPDATE[args.storage] // 2 * nodes, "strip": list(strip),
                      "autotune": tune_summary(tuned)}))
    ens.close()
    return 0


def tune_summary(tuned):
    """The autotuner's candidates as labels with their ms per step: tile geometries "rows x npt", and on
    the three-step strips "<staging>/<blocks per SM>b/<shared-memory KB>k" (staging "s0": none, "s1": one
    row in shared memory, "r1": one row in registers, "g": the generic-width kernel)."""
    if tuned is None:
        return None

    def label(c):
        if c["strip_blocks_per_sm"] > 0:
            st = {0: "g", 1: "s0", 2: "s1", 3: "r1"}[c["strip_stage"]]
            return f"{st}/{c['strip_blocks_per_sm']}b/{c['strip_smem_kb']}k"
        return f"{c['tile_rows']}x{c['nodes_per_thread']}"

    cands = tuned.get("candidates", [])
    out = {"tile_rows": tuned["tile_rows"], "nodes_per_thread": tuned["nodes_per_thread"],
           "autotune_ms_per_step": {label(c): round(c["ms_per_step"], 4) for c in cands}}
    if 0 <= tuned.get("chosen", -1) < len(cands):
        out["chosen"] = label(cands[tuned["chosen"]])
    return out


def _oracle_run(cases):
    """The oracle on `cases`, run after every timed GPU region so that no host work overlaps one."""
    from oracle import lbm as olbm

    t0 = time.perf_counter()
    res = olbm.run(cases)
    return res, time.perf_counter() - t0


def _oracle_cases(specs):
    from oracle import lbm as olbm

    return [olbm.Case(s.kind, s.nx, s.ny, s.steps, s.nu, s.u0, amp2=s.amp2, amp3=s.amp3, u_ref=s.u_ref,
                      cyl_cx=s.cyl_cx, cyl_cy=s.cyl_cy, cyl_r=s.cyl_r, ramp_steps=s.ramp_steps,
                      qoi_every=100 if s.steady_tol > 0 else 0, steady_tol=s.steady_tol,
                      pert=tuple(s.pert), obstacle_bc=s.obstacle_bc, inout_bc=s.inout_bc) for s in specs]


def _rel(a, b):
    import numpy as np

    a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _mc_against_sc(ens, w_mc, mc_fields, torch):
    """Sec. 8.2's comparison of Monte Carlo with stochastic collocation, on the 4-D workload: the
    reference is the 5^4 tensor Gauss-Legendre collocation of the same set-up (total degree 4), run
    with the same storage; the Monte Carlo mean and standard-deviation fields of N samples (disjoint
    blocks of the seeded sequence, up to 32 blocks per N) are compared with it in relative L2, and
    the RMS error over the blocks is fitted against N (Monte Carlo converges as N^-1/2)."""
    import numpy as np

    from paper_2508_13867_gb300 import workloads as W

    w_sc = W.tgv256_gpc4d(n=w_mc.base.nx, steps=w_mc.base.steps, storage=w_mc.storage)
    ens.setup(w_sc)
    smp = ens.ensemble_samples(w_sc)
    rsc = ens.run_batch(smp, storage=w_sc.storage, fields_dtype="f32")
    mean_sc, var_sc = ens.stats(ens.project(rsc["fields"]))
    del rsc
    ens.setup(w_mc)
    ref_mean = mean_sc[:-1]
    ref_std = torch.sqrt(var_sc[:-1])
    S = mc_fields.shape[0]
    out = {"reference": f"5^4 Gauss-Legendre collocation, total degree 4, {w_sc.storage} storage",
           "n": [], "blocks": [], "mean_rel_l2": [], "std_rel_l2": []}
    n = 16
    while n <= S:
        blocks = min(S // n, 32)
        em, es = [], []
        for b in range(blocks):
            m = mc_fields[b * n:(b + 1) * n, :-1].double()
            mu = m.mean(0)
            sd = m.std(0, unbiased=True)
            em.append(float(torch.linalg.norm(mu - ref_mean) / torch.linalg.norm(ref_mean)))
            es.append(float(torch.linalg.norm(sd - ref_std) / torch.linalg.norm(ref_std)))
            del m, mu, sd
        out["n"].append(n)
        out["blocks"].append(blocks)
        out["mean_rel_l2"].append(float(np.sqrt(np.mean(np.square(em)))))
        out["std_rel_l2"].append(float(np.sqrt(np.mean(np.square(es)))))
        n *= 2
    sel = [i for i, b in enumerate(out["blocks"]) if b >= 4]
    if len(sel) >= 2:
        x = np.log([out["n"][i] for i in sel])
        out["slope_mean"] = float(np.polyfit(x, np.log([out["mean_rel_l2"][i] for i in sel]), 1)[0])
        out["slope_std"] = float(np.polyfit(x, np.log([out["std_rel_l2"][i] for i in sel]), 1)[0])
        out["slope_fit_over_n"] = [out["n"][i] for i in sel]
    return out


def bench_workload(args):
    """The other workloads of the method, one JSON line each: throughput of the whole pass and,
    where an oracle reference is affordable, the error of the statistics against it."""
    import numpy as np
    import torch

    from oracle import lbm as olbm
    from oracle import uq as ouq
    from paper_2508_13867_gb300 import build as lib_build

    lib_build.build()
    olbm.build()
    from paper_2508_13867_gb300 import uqlb as U
    from paper_2508_13867_gb300 import workloads as W
    from paper_2508_13867_gb300.ensemble import Ensemble, sample_struct

    ens = Ensemble(0)
    line = {"workload": args.workload, "storage": args.storage, "unit": UNIT}
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    if args.workload in ("tgv64_gpc", "tgv512_mc4d", "cylinder"):
        if args.workload == "tgv64_gpc":
            w = W.tgv64_gpc()
        elif args.workload == "tgv512_mc4d":
            w = W.tgv512_mc4d(n=args.n or 512, steps=args.time_steps_full or 2000, n_mc=args.n_mc or 4096,
                              storage=args.storage)
        else:
            w = W.cylinder_gpc(nd=args.nd, storage=args.storage, bc=args.obstacle_bc, inout=args.inout_bc)
        if args.workload == "tgv64_gpc":
            w.storage = args.storage if args.storage != "f32" else "f64"
        line["storage"] = w.storage
        ens.setup(w)
        smp = ens.ensemble_samples(w)
        specs = [W.SampleSpec(s.kind, s.nx, s.ny, s.steps, s.nu, s.u0, s.amp2, s.amp3, s.u_ref, s.cyl_cx, s.cyl_cy,
                              s.cyl_r, s.ramp_steps, s.steady_tol, s.steady_checks, tuple(s.pert), s.obstacle_bc,
                              s.inout_bc)
                 for s in smp]
        n_oracle = args.oracle_samples if args.oracle_samples >= 0 else (64 if args.workload == "tgv512_mc4d" else 4)
        sub = list(range(min(len(specs), n_oracle)))
        fd = "f64" if w.storage == "f64" else "f32"
        qe = w.qoi_every

        def run():
            r = ens.run_batch(smp, storage=w.storage, fields_dtype=fd, qoi_every=qe, mode=args.mode, scheme=args.scheme)
            if w.method == "gpc":
                c = ens.project(r["fields"])
                m, v = ens.stats(c)
            else:
                m, v = ens.stats(r["fields"], ddof=1)
            return r, m, v

        ms, (r, mean, var) = timed(run, args.steps)
        upd = sum(int(qq[U.UQLB_QOI_STEPS]) for qq in r["qoi"].cpu().numpy()) * smp[0].nx * smp[0].ny
        line.update({"samples": len(smp), "lattice": [smp[0].nx, smp[0].ny], "time_to_stats_s": ms / 1e3,
                     "value": upd / (ms / 1e3) / 1e6, "mode": args.mode, "scheme": args.scheme})
        # further storage formats of the same ensemble (compared with the same oracle subset)
        extra = {}
        for spec in [x for x in args.storages.split(",") if x and x != w.storage]:
            st, _, rounding = spec.partition(":")

            def run_st(st=st, rounding=rounding or "auto"):
                rr = ens.run_batch(smp, storage=st, fields_dtype="f32", rounding=rounding)
                return rr, ens.stats(rr["fields"], ddof=1) if w.method == "mc" else ens.stats(ens.project(rr["fields"]))
            ms_st, (rr, _) = timed(run_st, 1)
            extra[spec] = {"time_to_stats_s": ms_st / 1e3, "value": upd / (ms_st / 1e3) / 1e6,
                           "fields": rr["fields"][sub].double().cpu().numpy()}
            del rr
        # plain per-sample FP64 comparator on a subset, scaled by the sample count (halfway
        # bounce-back only)
        if args.plain_samples > 0 and not any(s.obstacle_bc or s.inout_bc for s in smp):
            psub = [smp[i] for i in range(min(len(smp), args.plain_samples))]
            pms, _ = timed(lambda: ens.run_plain_f64(psub, fields=True), 1)
            line["plain_f64_time_to_stats_s"] = pms / 1e3 * len(smp) / len(psub)
            line["speedup_vs_plain_f64"] = line["plain_f64_time_to_stats_s"] / line["time_to_stats_s"]
        mc_sc = None
        if args.workload == "tgv512_mc4d" and args.mc_vs_sc:
            mc_sc = _mc_against_sc(ens, w, r["fields"], torch)
        g_fields = r["fields"][sub].double().cpu().numpy()
        q_all = r["qoi"].cpu().numpy()
        del r
        line["steps_run"] = [int(v) for v in q_all[:, U.UQLB_QOI_STEPS]]
        geo = U.uqlb_last_run_geometry(ens.ctx)
        line["ran_as"] = {1: "one_step", 3: "two_step_tiles", 4: "two_step_strips", 5: "groups", 6: "three_step_strips",
                          7: "cluster"}[geo[0]]
        line["geometry"] = list(geo[1:])
        if not sub:
            if mc_sc is not None:
                line["mc_vs_sc"] = mc_sc
            print(json.dumps(line))
            ens.close()
            return 0
        ref, oracle_s = _oracle_run(_oracle_cases([specs[i] for i in sub]))
        m_ref = np.stack([np.concatenate([q.u.ravel(), q.v.ravel(), [q.k_final]]) for q in ref])
        line["oracle_samples"] = len(sub)
        line["oracle_seconds"] = oracle_s
        line["host_work_overlapping_timed_regions"] = False
        if mc_sc is not None:
            line["mc_vs_sc"] = mc_sc
        line["field_rel_l2_worst_sample"] = max(_rel(g_fields[i, :-1], m_ref[i, :-1]) for i in range(len(sub)))
        if args.workload == "cylinder":
            q = q_all
            line["cd"] = q[:, U.UQLB_QOI_CD].tolist()
            line["steps_run"] = q[:, U.UQLB_QOI_STEPS].tolist()
            line["cd_oracle"] = [x.cd for x in ref]
            line["steps_oracle"] = [x.steps_run for x in ref]
            if len(sub) == len(smp):
                z, xi, a = ouq.tensor_grid([w.pts_per_dim], w.bounds)
                cd_o = np.array([[x.cd] for x in ref])
                c_o = ouq.gpc_coefficients(ouq.multi_indices(1, w.order), xi, a, cd_o)
                mo, vo = ouq.gpc_mean_var(c_o)
                c_g = ouq.gpc_coefficients(ouq.multi_indices(1, w.order), xi, a, q[:, [U.UQLB_QOI_CD]])
                mg, vg = ouq.gpc_mean_var(c_g)
                line["cd_mean_std"] = [float(mg[0]), float(np.sqrt(vg[0]))]
                line["cd_mean_std_oracle"] = [float(mo[0]), float(np.sqrt(vo[0]))]
        elif w.method == "mc":
            mu_r, var_r = ouq.mc_mean_var(m_ref, ddof=1)
            per = {w.storage: {"fields": g_fields, "value": line["value"], "time_to_stats_s": line["time_to_stats_s"]}}
            per.update(extra)
            line["precision"] = {}
            for st, d in per.items():
                gm, gv = ouq.mc_mean_var(d["fields"], ddof=1)
                line["precision"][st] = {
                    "value": d["value"], "time_to_stats_s": d["time_to_stats_s"],
                    "field_rel_l2_worst_sample": max(_rel(d["fields"][i, :-1], m_ref[i, :-1]) for i in range(len(sub))),
                    "subset_mean_rel_l2": _rel(gm[:-1], mu_r[:-1]),
                    "subset_std_rel_l2": _rel(np.sqrt(gv[:-1]), np.sqrt(var_r[:-1]))}
        else:
            z, xi, a = ouq.tensor_grid([w.pts_per_dim] * len(w.bounds), w.bounds)
            c_ref = ouq.gpc_coefficients(ouq.multi_indices(len(w.bounds), w.order), xi, a, m_ref)
            mr, vr = ouq.gpc_mean_var(c_ref)
            line["mean_rel_l2"] = _rel(mean.cpu().numpy(), mr)
            line["std_rel_l2"] = _rel(np.sqrt(var.cpu().numpy()), np.sqrt(vr))
    elif args.workload == "tgv_paper4d":
        # Sec. 8.3 study: ensembles at several resolutions n to T_max = 100 (Monte Carlo with N = n
        # samples, or the Smolyak grid), W1 of the pooled |u| values against the finest resolution
        # at t = 0.2, 0.4, ..., 1.0 T_max.  A snapshot in which a sample has gone unstable (rho <= 0
        # or a non-finite velocity at some node) gets no distance: its fields are not a solution.
        res_list = [int(x) for x in args.resolutions.split(",")]
        ref_n = max(res_list)
        fracs = [0.2, 0.4, 0.6, 0.8, 1.0]
        snaps, unstable, timing = {}, {}, {}
        for n in res_list:
            pconv = U.uqlb_unit_converter(n, 1.6 / n, 40.0 * n)
            total = int(round(args.t_max / pconv["dt"]))
            w = W.tgv_paper4d(n, pconv["tau"], pconv["u_lattice"], total, sampling=args.sampling,
                              storage=args.storage)
            ens.setup(w)
            base = ens.ensemble_samples(w)
            marks = [int(round(f * total)) for f in fracs]
            snaps[n], unstable[n] = [], []
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            prev = 0
            for m in marks:
                for smp_ in base:
                    smp_.steps = m
                r = ens.run_batch(base, storage=args.storage, fields_dtype="f32", start_step=prev)
                snaps[n].append(r["fields"].clone())
                unstable[n].append(r["qoi"][:, U.UQLB_QOI_STATUS] == U.UQLB_ERR_UNSTABLE)
                prev = m
            e1.record(stream)
            torch.cuda.synchronize()
            sec = e0.elapsed_time(e1) / 1e3
            upd = len(base) * (n - 1) ** 2 * total
            unstable[n] = [int(u.sum().item()) for u in unstable[n]]
            timing[n] = {"samples": len(base), "lattice": n - 1, "steps": total, "tau": pconv["tau"],
                         "seconds": sec, "value": upd / sec / 1e6, "seconds_per_sample": sec / len(base),
                         "unstable_samples": dict(zip([f * args.t_max for f in fracs], unstable[n]))}
        line["sampling"] = args.sampling
        line["resolutions"] = timing
        line["w1_vs_finest"] = {}
        for n in res_list:
            if n == ref_n:
                continue
            row = []
            for k in range(len(fracs)):
                d, bound, nf = ens.w1_speed(snaps[n][k], (n - 1) ** 2, snaps[ref_n][k], (ref_n - 1) ** 2)
                ok = unstable[n][k] == 0 and unstable[ref_n][k] == 0 and nf == (0, 0)
                row.append({"t": fracs[k] * args.t_max, "w1": d if ok else None, "bound": bound if ok else None,
                            "unstable_samples": unstable[n][k], "nonfinite_speeds": nf[0]})
            line["w1_vs_finest"][str(n)] = row
        line["value"] = timing[ref_n]["value"]
    elif args.workload == "cylinder_uq_compare":
        # Sec. 8.1 comparison of UQ methods on the cylinder at nd nodes per diameter: MC and QMC
        # (Halton) with N = 10 ... 100 samples against the SC-gPC reference (11 Gauss-Legendre
        # points, order 5), mean and standard deviation of the steady C_D, plus the deterministic
        # C_D at the nominal inflow.  MC and QMC sets of size N are prefixes of one sequence, so
        # one batch holds every sample.
        n_list = [int(x) for x in args.compare_n.split(",")]
        n_max = max(n_list)
        st = args.storage if args.storage != "f32" else "f64"
        mk = lambda method, n: W.cylinder_uq(args.nd, method=method, n=n, spread=args.inflow_spread, storage=st,  # noqa: E731
                                             bc=args.obstacle_bc, inout=args.inout_bc)
        w_sc, w_mc, w_qmc = mk("gpc", 11), mk("mc", n_max), mk("qmc", n_max)
        groups = {}
        for name, w in (("sc", w_sc), ("mc", w_mc), ("qmc", w_qmc)):
            ens.setup(w)
            groups[name] = ens.ensemble_samples(w)
        det = W.channel(args.nd, steps=w_sc.base.steps, steady_tol=w_sc.base.steady_tol, bc=args.obstacle_bc,
                        inout=args.inout_bc)
        det.steady_checks = w_sc.base.steady_checks
        smp = groups["sc"] + groups["mc"] + groups["qmc"] + [sample_struct(det)]
        ms, r = timed(lambda: ens.run_batch(smp, storage=st, fields=False, qoi_every=100), 1)
        q = r["qoi"]
        cd = q[:, U.UQLB_QOI_CD].contiguous()
        o_sc, o_mc, o_qmc = 0, len(groups["sc"]), len(groups["sc"]) + len(groups["mc"])
        ens.setup(w_sc)
        m_sc, v_sc = ens.stats(ens.project(cd[o_sc:o_mc].reshape(-1, 1)))
        ref = (float(m_sc[0]), float(v_sc[0]) ** 0.5)
        table = {"sc_gpc": {"n": len(groups["sc"]), "order": w_sc.order, "mean": ref[0], "std": ref[1]}}
        for name, off, init in (("mc", o_mc, lambda n: ens.init_mc(n, w_mc.seed)), ("qmc", o_qmc, ens.init_qmc)):
            rows = []
            for n in n_list:
                init(n)
                m, v = ens.stats(cd[off:off + n].reshape(-1, 1), ddof=1)
                mean, std = float(m[0]), float(v[0]) ** 0.5
                rows.append({"n": n, "mean": mean, "std": std, "rel_err_mean": abs(mean - ref[0]) / abs(ref[0]),
                             "rel_err_std": abs(std - ref[1]) / abs(ref[1])})
            table[name] = rows
        steps = q[:, U.UQLB_QOI_STEPS].cpu().numpy()
        status = q[:, U.UQLB_QOI_STATUS].cpu().numpy()
        upd = int(steps.sum()) * smp[0].nx * smp[0].ny
        line.update({"samples": len(smp), "lattice": [smp[0].nx, smp[0].ny], "storage": st,
                     "obstacle_bc": args.obstacle_bc, "inout_bc": args.inout_bc,
                     "inflow": [w_sc.bounds[0][0], w_sc.bounds[0][1]], "seconds": ms / 1e3,
                     "value": upd / (ms / 1e3) / 1e6, "steps_run": [int(steps.min()), int(steps.max())],
                     "samples_not_converged": int((steps >= w_sc.base.steps).sum()),
                     "unstable_samples": int((status == U.UQLB_ERR_UNSTABLE).sum()),
                     "cd_deterministic": float(cd[-1]), "cd_stats": table})
    elif args.workload in ("uneven", "uneven_channels"):
        # uneven_channels: the batch's 64 channel samples alone
        specs = W.uneven_batch()
        if args.workload == "uneven_channels":
            specs = [s for s in specs if s.kind == W.CHANNEL]
        smp = [sample_struct(s) for s in specs]
        tuned = ens.autotune(smp, storage=args.storage, trial_steps=8, scheme=args.scheme)
        ms, r = timed(lambda: ens.run_batch(smp, storage=args.storage, fields=False, scheme=args.scheme), args.steps)
        upd = sum(s.nx * s.ny * s.steps for s in specs)
        line.update({"samples": len(smp), "value": upd / (ms / 1e3) / 1e6, "batch_seconds": ms / 1e3,
                     "tile_geometry": tune_summary(tuned), "scheme": args.scheme,
                     "ran_as": {0: "auto", 1: "one_step", 3: "two_step_tiles", 4: "two_step_strips",
                                5: "groups", 6: "three_step_strips", 7: "cluster"}[U.uqlb_last_run_geometry(ens.ctx)[0]]})
        if args.plain_samples > 0:
            step = max(1, len(smp) // args.plain_samples)
            psub = smp[::step]
            pms, _ = timed(lambda: ens.run_plain_f64(psub, fields=False), 1)
            pupd = sum(s.nx * s.ny * s.steps for s in psub)
            line["plain_f64_seconds_scaled"] = pms / 1e3 * upd / pupd
            line["speedup_vs_plain_f64"] = line["plain_f64_seconds_scaled"] / line["batch_seconds"]
    print(json.dumps(line))
    ens.close()
    return 0


def bench_gpu(args):
    import numpy as np
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2508_13867_gb300 import build as lib_build

    lib_build.build()
    from paper_2508_13867_gb300 import uqlb as U
    from paper_2508_13867_gb300 import workloads as W
    from paper_2508_13867_gb300.ensemble import Ensemble, case_struct, opts_struct

    from paper_2508_13867_gb300 import shard

    w = W.tgv256_gpc4d(storage=args.storage if args.storage != "f64" else "f32")
    ens = Ensemble(local)
    ens.setup(w)
    smp = ens.ensemble_samples(w)
    S, K = len(smp), ens.num_terms
    F = 2 * w.base.nx * w.base.ny + 1
    upd_per_step = _updates(smp)
    # sample-level sharding: this rank's contiguous block, balanced by nodes x steps; the partial
    # coefficients of the blocks are summed by one all-reduce (the only exchange)
    lo, hi = shard.partition(shard.sample_costs(smp), world)[rank]
    block = smp[lo:hi]
    storage = w.storage
    stream = torch.cuda.current_stream()
    dev = f"cuda:{local}"
    fields = torch.empty((hi - lo, F), dtype=torch.float32, device=dev)
    qoi = torch.empty((hi - lo, U.UQLB_QOI_COLS), dtype=torch.float64, device=dev)
    coeffs = torch.empty((K, F), dtype=torch.float64, device=dev)
    out = {"fields": fields, "qoi": qoi}

    tuned = (ens.autotune(block, storage=storage, trial_steps=args.tune_steps, scheme=args.scheme)
             if args.tune_steps > 0 else None)

    def one_step():
        ens.run_batch(block, storage=storage, fields_dtype="f32", out=out, scheme=args.scheme)
        if world > 1:
            ens.project_block(fields, lo, coeffs)
            dist.all_reduce(coeffs, op=dist.ReduceOp.SUM)
        else:
            ens.project(fields, coeffs)
        return ens.stats(coeffs)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    loop_ms, loop_steps, launches = 0.0, 0, 0
    step_ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ms, st, la = U.uqlb_last_loop_time(ens.ctx)
        loop_ms += ms
        loop_steps += st
        # + the projection's launches (one per input dimension when sum-factorized) and the statistics
        n_proj = len(w.bounds) if world == 1 and U.uqlb_last_projection(ens.ctx) == 1 else 1
        launches += la + n_proj + 1
    ev0.record(stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * upd_per_step * args.steps / (total_ms / 1e3) / 1e6

    # roofline of the dominant kernel, from its event-timed loop.  One launch reads and writes
    # every population once (72 B per FP32 node); the two-step kernel advances two steps per launch.
    scheme, g_rows, g_npt = U.uqlb_last_run_geometry(ens.ctx)
    steps_per_launch = STEPS_PER_LAUNCH[scheme]
    kernel_name, ncu_name, kernel_version = STEP_KERNELS[scheme]
    nodes = (hi - lo) * w.base.nx * w.base.ny
    per_launch_bytes = BYTES_PER_UPDATE[storage] * nodes
    step_kernel_ms = loop_ms / max(loop_steps / steps_per_launch, 1)
    achieved = per_launch_bytes / (step_kernel_ms / 1e3) / 1e9
    peak, peak_kind = _peaks()
    traffic = read_traffic(ncu_name, storage, kernel_version)
    if traffic is not None and world > 1:
        traffic = int(traffic * (hi - lo) / S)

    # end to end through host buffers: one C call, tables in, statistics out (one GPU); the sharded
    # pass through the public calls with the statistics copied to the host (several GPUs)
    e2e = None
    if world > 1:
        mean_pin = torch.empty(F, dtype=torch.float64, pin_memory=True)
        var_pin = torch.empty(F, dtype=torch.float64, pin_memory=True)
        reps = max(1, min(args.steps, 3))
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(reps):
            mean_d, var_d = one_step()
            mean_pin.copy_(mean_d, non_blocking=True)
            var_pin.copy_(var_d, non_blocking=True)
            torch.cuda.synchronize()
        el = torch.tensor([(time.perf_counter() - t0) / reps], dtype=torch.float64, device=dev)
        dist.all_reduce(el, op=dist.ReduceOp.MAX)
        e2e_s = float(el.item())
        e2e = {"value": upd_per_step / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": (hi - lo) * (128 + 32 + 4),
               "d2h_bytes_per_step": 2 * F * 8, "seconds_per_step": e2e_s,
               "path": "sharded pass: uqlb_run_batch of the rank's block, uqlb_project_block, one NCCL all-reduce, "
                       "uqlb_stats, statistics copied to pinned host memory"}
    elif rank == 0:
        mean_h = np.zeros(F)
        var_h = np.zeros(F)
        case = case_struct(w)
        opts = opts_struct(storage, "f32", 0)
        nb = U.uqlb_uq_workspace_bytes(ens.ctx, case, opts)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        U.uqlb_run_uq_host(ens.ctx, case, opts, ws.data_ptr(), nb, mean_h, var_h, None, None, stream.cuda_stream)
        t0 = time.perf_counter()
        reps = max(1, min(args.steps, 3))
        for _ in range(reps):
            U.uqlb_run_uq_host(ens.ctx, case, opts, ws.data_ptr(), nb, mean_h, var_h, None, None, stream.cuda_stream)
        e2e_s = (time.perf_counter() - t0) / reps
        h2d = S * (128 + 32 + 4) + K * S * 8
        d2h = 2 * F * 8
        e2e = {"value": upd_per_step / e2e_s / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "seconds_per_step": e2e_s,
               "path": "uqlb_run_uq_host (one C call, host output buffers)"}
        del ws

    # comparator: plain per-sample FP64 path on a subset, time to the same gPC statistics
    plain = None
    if args.plain_samples > 0 and rank == 0:
        sub = smp[: args.plain_samples]
        res = ens.run_plain_f64(sub, qoi_every=0, fields=True)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        res = ens.run_plain_f64(sub, qoi_every=0, fields=True)
        t1.record(stream)
        torch.cuda.synchronize()
        plain_ms_sub = t0.elapsed_time(t1)
        plain_ms = plain_ms_sub * S / len(sub)
        ours_ms = total_ms / args.steps
        plain = {"time_to_stats_s": plain_ms / 1e3, "samples_timed": len(sub),
                 "extrapolated_to_samples": S, "batched_fp32_time_to_stats_s": ours_ms / 1e3,
                 "speedup": plain_ms / ours_ms,
                 "note": "plain path: one sample at a time, one FP64 launch per step, two lattices; "
                         "its time is linear in the samples, so the subset time is scaled by S / subset"}
        del res

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        mlups, el, upd, cores = run_oracle_slice(w, args.cpu_slice)
        cpu = {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"all 625 samples x {args.cpu_slice} of 2000 time steps ({upd:.3g} node updates, "
                         f"{el:.1f} s)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": storage,
                "data": "synthetic (seeded 4-D Taylor-Green ensemble)",
                "config": {"workload": "tgv256_gpc4d", "samples": S, "lattice": [256, 256], "time_steps": 2000,
                           "storage": storage, "statistics": "fp64", "gpc_terms": K,
                           "parallelism": (f"sample blocks x{world} (NCCL all-reduce of the partial gPC "
                                           "coefficients)" if world > 1 else "single GPU"),
                           "l2": "lattice arena 1.47 GB > L2 129 MB: each launch streams from HBM",
                           "scheme": {U.UQLB_SCHEME_ONE_STEP: "one_step", U.UQLB_SCHEME_TWO_STEP_TILES: "two_step_tiles",
                                      U.UQLB_SCHEME_TWO_STEP_STRIPS: "two_step_strips",
                                      U.UQLB_SCHEME_THREE_STEP_STRIPS: "three_step_strips"}[scheme],
                           "tile_geometry": tune_summary(tuned)},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                             "kernel": kernel_name, "time_steps_per_launch": steps_per_launch,
                             "algorithmic_bytes_per_launch": per_launch_bytes,
                             "bytes_per_update": per_launch_bytes / (nodes * steps_per_launch),
                             "bytes_per_update_one_step": BYTES_PER_UPDATE[storage],
                             "frac_at_one_step_bytes": achieved * steps_per_launch / peak,
                             "note": (f"achieved = the scheme's algorithmic bytes per launch ({BYTES_PER_UPDATE[storage]} B "
                                      f"per node: every population read and written once per launch, "
                                      f"{steps_per_launch} node update(s) per launch) / event-timed kernel time; "
                                      "frac_at_one_step_bytes counts the one-step scheme's "
                                      f"{BYTES_PER_UPDATE[storage]} B for every node update"),
                             "kernel_ms_per_launch": step_kernel_ms},
                "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
                "plain_f64": plain}
        print(json.dumps(line))
    ens.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-slice", type=int, default=40, help="oracle time steps per sample for cpu_baseline")
    ap.add_argument("--ref-slice", type=int, default=16, help="oracle time steps per sample per reference step")
    ap.add_argument("--plain-samples", type=int, default=16)
    ap.add_argument("--tune-steps", type=int, default=16, help="autotuner trial steps per geometry (0: off)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--kernel-only", action="store_true", help="small ensemble-run case for profiler captures")
    ap.add_argument("--samples", type=int, default=128)
    ap.add_argument("--time-steps", type=int, default=16)
    ap.add_argument("--lattice", type=int, default=0, help="kernel-only: lattice side N (0: the workload's 256)")
    ap.add_argument("--kernel-case", default="tgv", choices=["tgv", "cylinder"],
                    help="kernel-only: the 4-D Taylor-Green samples or channel samples of the cylinder workload (--nd)")
    ap.add_argument("--strip", default="0,0,0",
                    help="kernel-only: three-step strips' blocks per SM, staging option (1: none, 2: one row in shared memory, "
                         "3: one row in registers) and "
                         "shared-memory KB (0: tuned or default)")
    ap.add_argument("--kernel-autotune", action="store_true",
                    help="kernel-only: run the autotuner (--tune-steps) first and report its candidates")
    ap.add_argument("--storage", default="f32", choices=["f64", "f32", "f16", "bf16", "fx16"])
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--npt", type=int, default=0)
    ap.add_argument("--rounding", default="auto", choices=["auto", "nearest", "stochastic"])
    ap.add_argument("--scheme", default="auto",
                    choices=["auto", "one_step", "two_step", "two_step_tiles", "two_step_strips", "three_step_strips",
                             "cluster"],
                    help="time-stepping scheme (auto: two-step for periodic FP32/16-bit batches)")
    ap.add_argument("--mode", default="graph", choices=["graph", "persistent"],
                    help="kernel-only: one launch per step (CUDA graphs) or one cooperative launch per chunk")
    ap.add_argument("--workload", default="tgv256_gpc4d",
                    choices=["tgv256_gpc4d", "tgv64_gpc", "tgv512_mc4d", "cylinder", "cylinder_uq_compare", "uneven",
                             "uneven_channels", "tgv_paper4d"])
    ap.add_argument("--resolutions", default="8,16,32,64,128,256", help="tgv_paper4d: resolutions n")
    ap.add_argument("--t-max", type=float, default=100.0, help="tgv_paper4d: final physical time")
    ap.add_argument("--sampling", default="mc", choices=["mc", "smolyak"],
                    help="tgv_paper4d: Monte Carlo with N = n samples, or the level-3 Smolyak grid")
    ap.add_argument("--oracle-samples", type=int, default=-1,
                    help="oracle reference subset (other workloads; default 64 for tgv512_mc4d, else 4)")
    ap.add_argument("--no-mc-vs-sc", dest="mc_vs_sc", action="store_false",
                    help="tgv512_mc4d: skip the Monte Carlo error against the 5^4 collocation reference")
    ap.add_argument("--storages", default="", help="further storage formats to run on the same workload")
    ap.add_argument("--nd", type=int, default=20, help="cylinder: nodes per diameter")
    ap.add_argument("--obstacle-bc", default="halfway", choices=["halfway", "bouzidi"],
                    help="cylinder workloads: obstacle scheme")
    ap.add_argument("--inout-bc", default="face", choices=["face", "interpolated"],
                    help="cylinder workloads: inlet/outlet scheme")
    ap.add_argument("--compare-n", default="10,20,40,80,100", help="cylinder_uq_compare: MC/QMC sample counts")
    ap.add_argument("--inflow-spread", type=float, default=0.2, help="cylinder_uq_compare: relative inflow spread")
    ap.add_argument("--n", type=int, default=0, help="tgv512_mc4d: lattice size override")
    ap.add_argument("--n-mc", type=int, default=0, help="tgv512_mc4d: sample count override")
    ap.add_argument("--write-traffic", default="", help="ncu CSV of a --kernel-only capture: write the traffic file")
    ap.add_argument("--traffic-kernel", default="strip2_kernel")
    ap.add_argument("--traffic-command", default="")
    ap.add_argument("--time-steps-full", type=int, default=0, help="tgv512_mc4d: step count override")
    args = ap.parse_args()
    if args.write_traffic:
        ver = {k[1]: k[2] for k in STEP_KERNELS.values()}[args.traffic_kernel]
        print(write_traffic(args.write_traffic, args.traffic_kernel, args.storage, ver, args.samples,
                            args.traffic_command))
        return 0
    if args.impl == "reference":
        return bench_reference(args)
    if args.kernel_only:
        return bench_kernel_only(args)
    if args.workload != "tgv256_gpc4d":
        return bench_workload(args)
    return bench_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
