#!/usr/bin/env python
"""Benchmark of the stochastic multigrid SELM hot path on one GB300 (per rank).

Workload (one "step" = one Euler-Maruyama step of Algorithm 4, the whole hot
path): 3-D channel, 128^3 MAC grid on the unit box, periodic in x and y,
no-slip walls in z; 1024 particles uniform in the channel (2-cell wall
clearance) with fixed N(0,1) forces; dt = 1e-3.  Per step: Peskin spread,
MAC projection, FAC solve of A u = b to ||r|| <= 1e-10 ||b|| (FP32 smoothing
and transfers inside FP64 iterative refinement, FP64 coarsest solve),
2 stochastic FAC cycles of the thermal chain, projection, interpolation and
the particle update.

Metric: cell-cycles per second = 128^3 fine cells (all three velocity
components) x velocity V-cycles executed (solve + sample), divided by the
device time of the steps.  L2 (129 MB) is flushed between steps by writing a
256 MB buffer outside the timed events.

With --impl reference the FP64 CPU oracle is timed on the host cores instead
(one stochastic FAC cycle of the same 128^3 system per step).
"""

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stochastic-MG cells/s (frac of HBM peak); served solves/s + p99 vs plain form"
N_CELLS_EDGE = 128
N_PARTICLES = 1024
DT = 1e-3
SAMPLE_CYCLES = 2


def workload_config(n, npart, projection):
    return {
        "workload": f"3-D channel {n}^3 MAC grid (periodic x,y; no-slip walls z), {npart} particles, "
                    f"Euler-Maruyama dt={DT}, FAC solve to 1e-10 + {SAMPLE_CYCLES} stochastic cycles per step, "
                    f"FP32 smoothing/transfers with FP64 refinement and FP64 coarsest solve, "
                    f"projection={'MAC' if projection else 'none'}",
        "grid": n, "particles": npart, "dt": DT, "stochastic_cycles_per_step": SAMPLE_CYCLES,
        "tol": 1e-10, "levels": None, "l2": "flushed between steps (256 MB write, outside the timed events)",
        "unit_of_work": "cell-cycle = one fine cell (all 3 velocity components) through one V-cycle",
    }


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=N_CELLS_EDGE)
    p.add_argument("--particles", type=int, default=N_PARTICLES)
    p.add_argument("--no-projection", action="store_true")
    p.add_argument("--engine-level", type=int, default=0,
                   help="first multigrid level of the cluster-resident coarse engine (0 = automatic)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="headline workload only: no covariance, composite or 64^2 sub-records")
    p.add_argument("--workload", default="channel128", choices=["channel128", "batched", "served", "composite", "decorrelation", "mac"],
                   help="channel128: the headline line; batched: 64 uneven systems, batched vs plain; "
                        "served: Poisson request stream, served vs plain per-request")
    p.add_argument("--comp-n", type=int, default=256, help="composite workload: base cells per axis")
    p.add_argument("--comp-k", type=int, default=32, help="composite workload: refined base rows")
    p.add_argument("--mac-n", type=int, default=64, help="staggered composite workload: base cells per axis")
    p.add_argument("--mac-k", type=int, default=8, help="staggered composite workload: refined base rows")
    p.add_argument("--systems", type=int, default=64)
    p.add_argument("--requests", type=int, default=5000)
    p.add_argument("--rate", type=float, default=200.0)
    p.add_argument("--slots", type=int, default=12)
    p.add_argument("--budget-gb", type=float, default=32.0)
    p.add_argument("--serve-persistent", type=int, default=0,
                   help="served workload: continuous batching through the persistent batched launch (1) "
                        "or shared per-phase graph launches (0)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle timing (spawned process, one thread)
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import os, sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
from oracle import grid, multigrid, philox
n = {n}
s = grid.velocity_system(n, 3)
co = multigrid.Coarsest(s)
import selm_inputs
z = selm_inputs.fields(s.shapes(0), seed=1, scale=1e-2)
zero = s.zeros(0)
times = []
for k in range({reps}):
    t = time.perf_counter()
    multigrid.fac_cycle(s, z, zero, philox.PhiloxNoise(0, 0, k), 1.0, coarsest=co)
    times.append(time.perf_counter() - t)
print(json.dumps(times))
"""


def run_oracle_cycles(n, reps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET.format(root=ROOT, n=n, reps=reps)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def whole_job(seconds, units, world, device):
    """Whole-job figures of a replica run: the units every rank processed,
    summed, over the slowest rank's time (max over ranks).  With one rank,
    the rank's own figures."""
    if world == 1:
        return float(seconds), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def run_oracle_replicas(n, procs):
    """`procs` single-thread oracle processes at once, each timing one
    stochastic FAC cycle; returns the wall time from the first start to the
    last finish of the timed cycles (each process reports its own interval)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ORACLE_SNIPPET_WALL.format(root=ROOT, n=n)
    ps = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True) for _ in range(procs)]
    spans = []
    for p in ps:
        out, _ = p.communicate()
        if p.returncode != 0:
            return None
        spans.append(json.loads(out.strip().splitlines()[-1]))
    return max(b for _, b in spans) - min(a for a, _ in spans)


ORACLE_SNIPPET_WALL = r"""
import os, sys, time, json
sys.path.insert(0, {root!r})
from oracle import grid, multigrid, philox
import selm_inputs
n = {n}
s = grid.velocity_system(n, 3)
co = multigrid.Coarsest(s)
z = selm_inputs.fields(s.shapes(0), seed=1, scale=1e-2)
zero = s.zeros(0)
t0 = time.time()
multigrid.fac_cycle(s, z, zero, philox.PhiloxNoise(0, 0, 0), 1.0, coarsest=co)
print(json.dumps([t0, time.time()]))
"""


def cpu_baseline(n, all_cores=True):
    times = run_oracle_cycles(n, 1)
    t = times[0]
    out = {"value": n ** 3 / t, "unit": "cells/s", "cores": 1, "kind": "oracle",
           "sample": f"one stochastic FAC cycle (Algorithm 1 around the V-cycle of Algorithm 3) of the FP64 "
                     f"numpy oracle on the {n}^3 velocity system, single thread, {t:.1f} s",
           "cpu_model": cpu_model()}
    if all_cores:
        procs = os.cpu_count() or 1
        wall = run_oracle_replicas(n, procs)
        if wall:
            out["all_cores"] = {"value": procs * n ** 3 / wall, "unit": "cells/s", "cores": procs,
                                "sample": f"{procs} single-thread oracle processes at once, one stochastic FAC "
                                          f"cycle of the {n}^3 system each (independent replicas), "
                                          f"{wall:.1f} s from the first start to the last finish"}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    n = args.n
    times = run_oracle_cycles(n, args.warmup + args.steps)
    timed = times[args.warmup:]
    total = sum(timed)
    value = n ** 3 * len(timed) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n, args.particles, not args.no_projection),
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
                         "sample": f"each step: one stochastic FAC cycle of the {n}^3 FP64 oracle, single thread"},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, device_index):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="selm_clocks_", suffix=".csv")
        os.close(fd)
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Sources that define the kernels of the uniform-grid path (the profiled ones).
PROFILED_SOURCES = ["selm_kernels.cu", "selm_coarse.cu", "selm_coarse.h", "selm_devmath.h", "selm_internal.h",
                    "selm_launch.h", "selm_pdl.h"]


# The composite-grid kernels add their own source to those.
COMPOSITE_SOURCES = PROFILED_SOURCES + ["selm_composite.cu"]


def kernel_source_sha(sources=None):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1003_2680_gb300", "csrc")
    for name in sources or PROFILED_SOURCES:
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def composite_ncu_traffic():
    """Per-launch DRAM bytes of the profiled composite kernels (ncu on the
    192^3 case, scaled to the 256^3 workload by the cells processed), keyed by
    kernel, from summaries taken on the current source."""
    out = {}
    for name in ("composite_base_rb_192", "composite_patch_192", "composite_residual_df_192",
                 "composite_galerkin_residual_256", "composite_coarse_colour_256"):
        path = os.path.join(ROOT, "profiles", name + ".md")
        if not os.path.exists(path):
            continue
        text = open(path).read()
        m_k = re.search(r"^# `([A-Za-z0-9_]+)`", text, re.M)
        m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
        m_tr = re.search(r"traffic_bytes_per_launch_256:\s*([0-9.eE+]+)", text)
        if m_k and m_sha and m_tr and m_sha.group(1) == kernel_source_sha(COMPOSITE_SOURCES):
            out[m_k.group(1)] = float(m_tr.group(1))
    return out


def ncu_traffic(kernel_class, n):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel_class}_{n}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_tr or m_sha.group(1) != kernel_source_sha():
        return None
    return float(m_tr.group(1))


def pass_bytes(e, sizes, ncols):
    """Algorithmic bytes of one colour pass over the components of a level:
    the pass reads every unknown of its level once (the neighbours of the
    updated colour), reads b and writes v at the updated sites,
    e * (N_level + 2 N_colour) per component present in the pass."""
    total = 0.0
    for q in range(max(ncols)):
        total += sum(e * (n + 2 * n / nc) for n, nc in zip(sizes, ncols) if q < nc)
    return total


def system_sizes(S, h, system, lev):
    ncomp = S.selm_mg_ncomp(h, system)
    out = []
    for c in range(ncomp):
        (nx, ny, nz), _, _ = S.selm_mg_layout(h, system, lev, c)
        out.append(nx * ny * nz)
    return out


def fine_bytes_per_launch(S, h):
    """One red-black colour launch on the finest velocity level: reads all of
    v and b at half the sites, writes v at half the sites."""
    e = S.selm_mg_inner_bytes(h)
    N = sum(system_sizes(S, h, 0, 0))
    return e * (N + 2 * N / 2)


def coarse_bytes_per_vcycle(S, h, system, sweeps=4):
    """Algorithmic bytes of the Galerkin levels of one V-cycle of a system
    (every colour pass of every sweep; colour counts 12, or 8 for a component
    whose wall axis is vertex-type)."""
    e = S.selm_mg_inner_bytes(h)
    levels = S.selm_mg_levels(h, system)
    total = 0.0
    for lev in range(1, levels - 1):
        sizes = system_sizes(S, h, system, lev)
        ncols = [12] * len(sizes)
        if system == 0 and len(sizes) > 1:
            ncols[-1] = 8
        total += sweeps * pass_bytes(e, sizes, ncols)
    return total


# Byte model of the hot path per unknown-cycle (3-D, FP32 inner cycles, noise
# drawn in registers): a red+black sweep fused into one pass reads z and r and
# writes z (12 B, 4 sweeps per cycle); residual + restriction 8.5 B;
# prolongation + correction 8.5 B; so 65 B per unknown of a level per V-cycle,
# x 8/7 for the coarse levels, + 40 B of FP64 refinement (residual: read z, b
# (FP64), write r (FP32); update: read z, delta, write z) = 114 B.
MODEL_SWEEP_B = 12.0
MODEL_LEVEL_B = 65.0
MODEL_REFINE_B = 40.0
MODEL_CYCLE_B = 114.0


def level_unknowns(S, h, system):
    return [sum(system_sizes(S, h, system, lev)) for lev in range(S.selm_mg_levels(h, system))]


def model_coarse_bytes_per_vcycle(S, h, system):
    """The byte model's share of one V-cycle on the levels below the finest:
    65 B (x e/4) per unknown of every coarse level (sweeps and transfers)."""
    e = S.selm_mg_inner_bytes(h)
    return MODEL_LEVEL_B * (e / 4.0) * sum(level_unknowns(S, h, system)[1:])


def model_fine_bytes_per_colour_launch(S, h):
    """Half of a fused red+black sweep of the finest velocity level: 12 B (x e/4)
    per unknown-sweep, two colour launches per sweep."""
    e = S.selm_mg_inner_bytes(h)
    return 0.5 * MODEL_SWEEP_B * (e / 4.0) * level_unknowns(S, h, 0)[0]


# ---------------------------------------------------------------------------
# main GPU arm
# ---------------------------------------------------------------------------
def run_batched(args):
    """64 independent 3-D channel systems, edges drawn from {32,48,64,96,128},
    64..2048 particles (log-uniform), kT ~ U[0.5, 2], seed i.  The batched
    form (persistent launch per FAC cycle, or per-system graphs; the autotuner
    keeps the faster) against the plain per-instance method run one system
    after another and run on 16 concurrent streams."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_1003_2680_gb300 import _build
    _build.build()
    from paper_1003_2680_gb300 import selm as S
    import selm_inputs

    nsys = args.systems
    edges = selm_inputs.batched_edges(nsys, seed=0)
    rng = np.random.default_rng([0, 505])
    nps = [int(round(x)) for x in np.exp(rng.uniform(np.log(64), np.log(2048), size=nsys))]
    kTs = [float(x) for x in rng.uniform(0.5, 2.0, size=nsys)]
    descs = [S.make_desc(dim=3, n=e, kT=kT, precision=S.SELM_FP32_REFINE64, seed=i, instance=i, max_particles=2048)
             for i, (e, kT) in enumerate(zip(edges, kTs))]
    X0 = [selm_inputs.particles(npart, 3, e, seed=i) for i, (npart, e) in enumerate(zip(nps, edges))]
    F0 = [selm_inputs.forces(npart, 3, seed=i) for i, npart in enumerate(nps)]
    cells = [e ** 3 for e in edges]
    steps = args.steps

    def timed(fn, nsteps):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = [fn() for _ in range(nsteps)]
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3, out

    # plain: one system after the other through selm_mg_step
    handles = [S.selm_mg_create(d) for d in descs]
    Xp = [torch.tensor(x, device="cuda") for x in X0]
    Fp = [torch.tensor(f, device="cuda") for f in F0]

    def plain_step():
        cyc = 0
        for i, h in enumerate(handles):
            S.selm_mg_step(h, Xp[i], Fp[i], DT, 1, SAMPLE_CYCLES)
            cyc += cells[i] * (S.selm_mg_stats(h)[0] + SAMPLE_CYCLES)
        return cyc

    plain_step()
    X_plain = [x.cpu().numpy() for x in Xp]   # after one step from X0 (the accuracy check)
    for _ in range(max(0, args.warmup - 3)):
        plain_step()
    t_plain, cyc_plain = timed(plain_step, steps)

    # plain on 16 concurrent streams (host threads), the same handles
    nstreams = 16
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    Xm = [torch.tensor(x, device="cuda") for x in X0]

    def worker(w):
        st = streams[w]
        for i in range(w, nsys, nstreams):
            S.selm_mg_step(handles[i], Xm[i], Fp[i], DT, 1, SAMPLE_CYCLES, stream=st.cuda_stream)
        st.synchronize()

    torch.cuda.synchronize()
    with ThreadPoolExecutor(nstreams) as ex:
        list(ex.map(worker, range(nstreams)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        with ThreadPoolExecutor(nstreams) as ex:
            list(ex.map(worker, range(nstreams)))
    torch.cuda.synchronize()
    t_multi = time.perf_counter() - t0
    for h in handles:
        S.selm_mg_destroy(h)
    torch.cuda.synchronize()

    forms = {}
    for form in ("persistent", "graphs"):
        b = S.selm_batch_create(descs)
        chosen = S.selm_batch_autotune(b)
        tuned = S.selm_batch_info(b)
        S.selm_batch_set_persistent(b, 1 if form == "persistent" else 0)
        Xb = [torch.tensor(x, device="cuda") for x in X0]
        Fb = [torch.tensor(f, device="cuda") for f in F0]

        def batch_step():
            cy = S.selm_batch_step(b, Xb, Fb, DT, 1, SAMPLE_CYCLES)
            return sum(c * (max(cy) + SAMPLE_CYCLES) for c in cells)

        batch_step()
        x_first = [x.cpu().numpy() for x in Xb]
        for _ in range(max(0, args.warmup - 3)):
            batch_step()
        launches0 = S.selm_kernel_launches()
        with ClockSampler(torch.cuda.current_device()) as clk:
            t_b, cyc_b = timed(batch_step, steps)
        launches = S.selm_kernel_launches() - launches0
        # equal accuracy: the batched trajectories against the plain per-instance ones
        # (both start from X0 and take warm-up + timed steps with the same counters)
        forms[form] = {"system_steps_per_s": nsys * steps / t_b, "cell_cycles_per_s": sum(cyc_b) / t_b,
                       "ms_per_step": 1e3 * t_b / steps, "gpu_launches": int(launches), "clocks": clk.summary(),
                       "tuned": tuned, "engine_cluster": chosen}
        if form == "persistent":
            forms[form]["phase_us_solve_cycle"] = _phase_summary(S.selm_batch_phase_times(b, S.SELM_BATCH_SOLVE))
        forms[form]["x"] = x_first
        S.selm_batch_destroy(b)
    # the trajectories of the batched forms and the plain form (same steps, same counters)
    def pdiff(a, b_):   # minimum image along the periodic axes (x, y)
        d = a - b_
        d[:, :2] = (d[:, :2] + 0.5) % 1.0 - 0.5
        return d

    acc = {}
    for form in forms:
        xs = forms[form].pop("x")
        acc[form] = max(float(np.linalg.norm(pdiff(a, p_)) / max(np.linalg.norm(pdiff(p_, x0)), 1e-300))
                        for a, p_, x0 in zip(xs, X_plain, X0))
    best = max(forms, key=lambda k: forms[k]["system_steps_per_s"])
    line = {
        "metric": "batched stochastic-MG: system-steps/s and cell-cycles/s, batched vs plain per-instance",
        "value": forms[best]["system_steps_per_s"], "unit": "system-steps/s", "higher_is_better": True,
        "n_gpus": 1, "steps": steps, "warmup": args.warmup, "data": "synthetic", "dtype": "f32+f64",
        "config": {"workload": f"{nsys} independent 3-D channel systems, edges from {{32,48,64,96,128}}, "
                               f"64-2048 particles, kT in [0.5,2], one Euler-Maruyama step (solve to 1e-10 + "
                               f"{SAMPLE_CYCLES} stochastic cycles) per system per step",
                   "edges": edges, "best_form": best},
        "batched": forms,
        "plain": {"system_steps_per_s": nsys * steps / t_plain, "cell_cycles_per_s": sum(cyc_plain) / t_plain,
                  "ms_per_step": 1e3 * t_plain / steps},
        "plain_16_streams": {"system_steps_per_s": nsys * steps / t_multi, "ms_per_step": 1e3 * t_multi / steps,
                             "note": "the same handles stepped from 16 host threads, one CUDA stream each "
                                     "(wall clock)"},
        "speedup_steps": {"vs_plain": forms[best]["system_steps_per_s"] / (nsys * steps / t_plain),
                          "vs_plain_16_streams": forms[best]["system_steps_per_s"] / (nsys * steps / t_multi)},
        "equal_accuracy": {"max_rel_position_difference_vs_plain_after_one_step": acc,
                           "note": "every system's positions after one step from the same state, relative to "
                                   "the step's displacement (minimum image); FP32 inner cycles (tolerance 1e-5). "
                                   "Longer trajectories decorrelate at this resolution: a rounding-level "
                                   "difference grows about 15x per step"},
        "gpu_launches": forms[best]["gpu_launches"],
    }
    print(json.dumps(line), flush=True)


def _phase_summary(ph):
    agg = {}
    for name, lev, us in ph:
        key = f"{name}_L{lev}"
        a = agg.setdefault(key, [0, 0.0])
        a[0] += 1
        a[1] += us
    return {k: {"phases": v[0], "us": round(v[1], 1)} for k, v in sorted(agg.items(), key=lambda kv: -kv[1][1])}


def served_stream(nreq, rate, seed=0):
    """Poisson arrivals; 50% 2-D channels (edge 256..1024), 50% 3-D (edge 32..192);
    16..4096 particles (log-uniform); 1..20 Euler-Maruyama steps; own seed each."""
    import numpy as np
    rng = np.random.default_rng([seed, 606])
    t = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    reqs = []
    for i in range(nreq):
        if rng.uniform() < 0.5:
            dim, edge = 2, int(rng.choice([256, 384, 512, 768, 1024]))
        else:
            dim, edge = 3, int(rng.choice([32, 48, 64, 96, 128, 192]))
        npart = int(round(np.exp(rng.uniform(np.log(16), np.log(4096)))))
        reqs.append(dict(t=float(t[i]), dim=dim, n=edge, np=npart, steps=int(rng.integers(1, 21)), seed=1000 + i))
    return reqs


def run_served(args):
    import time as _time
    import numpy as np
    import torch
    from paper_1003_2680_gb300 import _build
    _build.build()
    from paper_1003_2680_gb300 import selm as S
    import selm_inputs

    reqs = served_stream(args.requests, args.rate)
    budget = int(args.budget_gb * (1 << 30))

    def serve(slots, batched=False, persistent=True):
        srv = S.selm_server_create_batched(budget, slots, persistent) if batched else S.selm_server_create(budget, slots)
        keep = []
        t0 = _time.perf_counter()
        for i, r in enumerate(reqs):
            delay = r["t"] - (_time.perf_counter() - t0)
            if delay > 0:
                _time.sleep(delay)
            X = np.ascontiguousarray(selm_inputs.particles(r["np"], r["dim"], r["n"], seed=r["seed"]))
            F = np.ascontiguousarray(selm_inputs.forces(r["np"], r["dim"], seed=r["seed"]))
            keep.append((X, F))
            desc = S.make_desc(dim=r["dim"], n=r["n"], kT=1.0, precision=S.SELM_FP32_REFINE64, seed=r["seed"],
                               instance=i, max_particles=r["np"], torch_allocator=False)
            S.selm_server_submit(srv, desc, X, F, DT, r["steps"], SAMPLE_CYCLES, user=i + 1)
        S.selm_server_drain(srv)
        res = S.selm_server_poll(srv, len(reqs) + 1)
        stats = S.selm_server_stats(srv)
        bstats = S.selm_server_batch_stats(srv) if batched else None
        S.selm_server_destroy(srv)
        lat = np.array([x["t_done"] - x["t_submit"] for x in res])
        span = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
        ok = all(x["status"] == 0 for x in res)
        busy = sum(x["t_done"] - x["t_admit"] for x in res)
        return dict(p50_ms=1e3 * float(np.percentile(lat, 50)), p99_ms=1e3 * float(np.percentile(lat, 99)),
                    requests_per_s=len(res) / span, solves_per_s=sum(r["steps"] for r in reqs) / span,
                    vcycles_per_s=sum(x["vcycles"] for x in res) / span, makespan_s=span,
                    mean_requests_in_service=busy / span,
                    peak_slots=stats["peak_slots"], peak_gb=stats["peak_bytes"] / 2 ** 30, all_ok=ok,
                    batched_steps=bstats["steps"] if bstats else None,
                    batch_rebuilds=bstats["rebuilds"] if bstats else None,
                    positions=[k[0].copy() for k in keep])

    torch.cuda.synchronize()
    plain = serve(1)
    streams = serve(args.slots)
    launches0 = S.selm_kernel_launches()
    served = serve(args.slots, batched=True, persistent=bool(args.serve_persistent))
    launches = S.selm_kernel_launches() - launches0
    # equal accuracy: every request's final positions, served vs plain (minimum
    # image along the periodic axes, relative to the request's displacement)
    worst, compared = 0.0, 0
    streams.pop("positions")
    for r, a, b_ in zip(reqs, served.pop("positions"), plain.pop("positions")):
        if r["steps"] > 1:   # longer trajectories decorrelate (rounding grows ~15x per step)
            continue
        compared += 1
        X0 = selm_inputs.particles(r["np"], r["dim"], r["n"], seed=r["seed"])
        def pd(u, v):
            d = u - v
            d[:, :-1] = (d[:, :-1] + 0.5) % 1.0 - 0.5
            return d
        worst = max(worst, float(np.linalg.norm(pd(a, b_)) / max(np.linalg.norm(pd(b_, X0)), 1e-300)))
    line = {
        "metric": "served solves/s + p99 vs plain form", "value": served["solves_per_s"], "unit": "solves/s",
        "form": "continuous batching: one batched Euler-Maruyama step of every admitted request per tick "
                "(" + ("persistent batched FAC launches" if args.serve_persistent else "shared per-phase graph launches")
                + "), requests retired and admitted between ticks",
        "higher_is_better": True, "n_gpus": 1, "data": "synthetic", "dtype": "f32+f64",
        "config": {"workload": f"{len(reqs)} requests, Poisson arrivals at {args.rate}/s; 50% 2-D channels "
                               f"(edge 256..1024), 50% 3-D (edge 32..192); 16..4096 particles; 1..20 steps; "
                               f"each step = FAC solve to 1e-10 + {SAMPLE_CYCLES} stochastic cycles",
                   "slots": args.slots, "budget_gb": args.budget_gb,
                   "solve": "one Euler-Maruyama step (one mobility solve) of one request"},
        "served": served, "plain": plain, "streams": streams,
        "speedup_solves": served["solves_per_s"] / plain["solves_per_s"],
        "speedup_vs_streams": served["solves_per_s"] / streams["solves_per_s"],
        "arms": {"plain": "one request at a time (one slot)",
                 "streams": f"{args.slots} slots, each request alone on its own stream (concurrency only)",
                 "served": f"{args.slots} slots, continuous batching"},
        "equal_accuracy": {"max_rel_position_difference_served_vs_plain": worst, "requests_compared": compared,
                           "note": "the one-step requests' positions, served against plain, relative to the "
                                   "displacement (minimum image); longer requests decorrelate chaotically at "
                                   "these resolutions (a rounding-level difference grows about 15x per step)"},
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)


def run_decorrelation(args):
    """Multigrid against Gauss-Seidel sampler (Section 5): lag correlations of a
    wall mode and a point probe, integrated autocorrelation times, time per
    iteration and independent variates per second, on the 2-D 64^2 FP64 grid
    and the 3-D 128^3 FP32-refined channel."""
    import numpy as np
    import torch
    from paper_1003_2680_gb300 import _build
    _build.build()
    from paper_1003_2680_gb300 import selm as S
    from paper_1003_2680_gb300 import decorrelation as D

    cases = [("2-D 64^2, FP64, 6 levels", 2, 64, S.SELM_FP64, 400),
             ("3-D 128^3, FP32 inner + FP64 refinement", 3, 128, S.SELM_FP32_REFINE64, 200)]
    out = {}
    launches = 0
    with ClockSampler(torch.cuda.current_device()) as clk:
        for name, dim, n, prec, k_gs in cases:
            m = S.SelmMG(dim=dim, n=n, precision=prec, seed=0, instance=0)
            h = m.h
            obs = {}
            for oname, phi in (("wall_mode", D.wall_mode(h, n)), ("point_probe", D.point_probe(h))):
                w = D.covariance_image(h, phi)
                r_mg = D.lag_correlations_mg(h, phi, 8, w)
                r_gs = D.lag_correlations_gs(h, phi, k_gs, w)
                obs[oname] = {
                    "mg": {"rho_1_to_4": [round(float(x), 6) for x in r_mg[1:5]],
                           "tau_int": D.integrated_time(r_mg), "lags_below_0.05": D.lags_below(r_mg)},
                    "gs": {"rho_at": {str(k): round(float(r_gs[k]), 6) for k in (1, 10, 50, 100, k_gs)},
                           "tau_int_lower_bound": D.integrated_time(r_gs),
                           "lags_below_0.05": D.lags_below(r_gs), "lags_computed": k_gs},
                }
            # time per iteration of each sampler (noise on, b = 0), events on the launching stream
            tot = S.selm_mg_layout(h, S.SELM_SYS_VELOCITY, 0, 0)[2]   # elements of the level field
            z = torch.zeros(tot, dtype=torch.float64, device="cuda")
            zero = torch.zeros_like(z)
            dt = torch.float32 if S.selm_mg_inner_bytes(h) == 4 else torch.float64
            v = torch.zeros(tot, dtype=dt, device="cuda")
            zv = torch.zeros_like(v)
            n_mg, n_gs = max(args.steps, 10) * 2, max(args.steps, 10) * 10
            for k in range(args.warmup):
                S.selm_mg_fac_cycle(h, S.SELM_SYS_VELOCITY, z, zero, k, 1)
                S.selm_mg_smooth(h, S.SELM_SYS_VELOCITY, 0, v, zv, 0, k, 1)
            torch.cuda.synchronize()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            l0 = S.selm_kernel_launches()
            a.record()
            for k in range(n_mg):
                S.selm_mg_fac_cycle(h, S.SELM_SYS_VELOCITY, z, zero, 100 + k, 1)
            b.record()
            for k in range(n_gs):
                S.selm_mg_smooth(h, S.SELM_SYS_VELOCITY, 0, v, zv, 0, 100 + k, 1)
            c.record()
            torch.cuda.synchronize()
            launches += S.selm_kernel_launches() - l0
            t_mg = a.elapsed_time(b) / 1e3 / n_mg
            t_gs = b.elapsed_time(c) / 1e3 / n_gs
            tau_mg = max(o["mg"]["tau_int"] for o in obs.values())
            tau_gs = max(o["gs"]["tau_int_lower_bound"] for o in obs.values())
            out[f"{dim}d_{n}"] = {
                "workload": name, "observables": obs,
                "mg_iteration_us": 1e6 * t_mg, "gs_sweep_us": 1e6 * t_gs,
                "mg_variates_per_s": 1.0 / (max(tau_mg, 1.0) * t_mg),
                "gs_variates_per_s_upper_bound": 1.0 / (tau_gs * t_gs),
                "mg_advantage_lower_bound": (tau_gs * t_gs) / (max(tau_mg, 1.0) * t_mg),
            }
            m.close()
    head = out["3d_128"]
    line = {
        "metric": "independent thermal variates/s of the multigrid sampler (1 / (tau_int x time per iteration))",
        "value": head["mg_variates_per_s"], "unit": "variates/s", "higher_is_better": True, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "data": "synthetic", "dtype": "f32+f64",
        "config": {"workload": "multigrid vs Gauss-Seidel sampler, wall mode and point probe of the x-velocity, "
                               "2-D 64^2 (FP64) and 3-D 128^3 (FP32 inner, FP64 refinement)",
                   "tau": "max over the two observables of 1 + 2 sum rho(k); Gauss-Seidel's is truncated at the "
                          "computed lags (a lower bound)",
                   "l2": "not flushed: consecutive iterations of one chain, as a sampler runs"},
        "samplers": out,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


COMPOSITE_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import composite as C, multigrid
from oracle.philox import PhiloxNoise
cg = C.CompositeGrid({n}, {K}, 3, ncomp=3)
co = multigrid.Coarsest(cg.base)
xi = [np.zeros(cg.size) for _ in range(3)]
zero = [np.zeros(cg.size) for _ in range(3)]
C.fac_cycle(cg, xi, zero, PhiloxNoise(0, 0, 0), 1.0, coarsest=co)
t = time.perf_counter()
C.fac_cycle(cg, xi, zero, PhiloxNoise(0, 0, 1), 1.0, coarsest=co)
print(json.dumps(time.perf_counter() - t))
"""


def composite_cpu_baseline(n, K):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = COMPOSITE_ORACLE_SNIPPET.format(root=ROOT, n=n, K=K)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    t = json.loads(out.stdout.strip().splitlines()[-1])
    cells = n ** 3 + (2 * n) ** 2 * 2 * K
    return {"value": cells / t, "unit": "cells/s", "cores": 1, "kind": "oracle",
            "sample": f"one stochastic composite FAC cycle of the FP64 oracle on the {n}^3 base with a "
                      f"{2 * n}x{2 * n}x{2 * K} patch (3 components), single thread, {t:.2f} s"}


def channel_covariance(S, h, n, nsamples=200):
    """Sample covariance of the handle's thermal chain on the 4^3 wall block
    (rows 0..3, every x-y translate) of each velocity component against the
    exact block of A^-1 (Fourier along x and y, sine transforms across the
    walls; the closed form the oracle is pinned against)."""
    from paper_1003_2680_gb300 import covariance as CV
    from tests import closed_forms as cf
    import numpy as np
    rows = (0, 1, 2, 3)
    res = CV.uniform_block(h, rows, nsamples=nsamples, nbatches=10)
    kinds = [("P", "P", "C"), ("P", "P", "C"), ("P", "P", "V")]
    exact = []
    for kd in kinds:
        nz = n - 1 if kd[2] == "V" else n
        cols = {}
        for r in rows:
            e = np.zeros((nz, n, n))
            e[r, 0, 0] = 1.0
            cols[r] = cf.spectral_solve(kd, n, 1.0 / n, e)
        sites = [(r, y, x) for r in rows for y in range(4) for x in range(4)]
        C = np.empty((64, 64))
        for j, (r2, y2, x2) in enumerate(sites):
            for i, (r1, y1, x1) in enumerate(sites):
                C[i, j] = cols[r2][r1, (y1 - y2) % n, (x1 - x2) % n]
        exact.append(C)
    out = CV.compare([res[c][0] for c in range(3)], [res[c][1] for c in range(3)], exact)
    out.update(samples=res[0][2], block="4^3 wall block (z rows 0..3) of each velocity component, averaged over "
                                         "all x-y translates", exact="A^-1 block, spectral closed form")
    return out


def golden_block(n, K):
    path = os.path.join(ROOT, "tests", "golden", f"composite_probe_cov_n{n}_K{K}.txt")
    if not os.path.exists(path):
        return None
    import numpy as np
    return np.loadtxt(path)


def composite_measure(S, n, K, steps, warmup, with_cpu, cov_samples=100):
    """The composite workload: a thermal sample = 2 stochastic composite FAC
    cycles of the persistent chain (256^3 base, bottom 32 rows refined by 2,
    three components, FP32 inner cycles with FP64 residual and coarsest solve).
    Returns the bench line as a dict."""
    import torch
    cycles_per_sample = SAMPLE_CYCLES
    c = S.selm_comp_create(S.make_comp_desc(3, n, K, ncomp=3, precision=S.SELM_FP32_REFINE64, seed=0, instance=0))
    N = S.selm_comp_size(c)
    e = S.selm_comp_inner_bytes(c)
    (fx, fy, fz), _, fsize = S.selm_comp_layout(c, 0, 0)
    (bx, by, bz), _, bsize = S.selm_comp_layout(c, 1, 0)
    cells = n ** 3 + fx * fy * fz
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(warmup):
        S.selm_comp_sample(c, cycles_per_sample)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = S.selm_kernel_launches()
    print(f"[bench] library kernel launches before the timed region: {launches0}", file=sys.stderr)
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record()
            S.selm_comp_sample(c, cycles_per_sample)
            ev[k][1].record()
        torch.cuda.synchronize()
    launches = S.selm_kernel_launches() - launches0
    t_total = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    value = cells * cycles_per_sample * steps / t_total

    # e2e: the same samples through the public call, each sample's 4^3 probe
    # block per component (x, y = 126..129; the two fine layers below and the two
    # base rows above the interface) read back to pinned host memory
    xi = torch.empty(N, dtype=torch.float64, device="cuda")
    probe_rows = []
    for comp in range(3):
        _, poff, _ = S.selm_comp_layout(c, 0, comp)
        _, boff, _ = S.selm_comp_layout(c, 1, comp)
        for m in (fz - 2, fz - 1):
            a = poff + (m * fy + 2 * 63) * fx
            probe_rows.append((a, a + 4 * fx))
        for r in (K, K + 1):
            a = boff + (r * by + 126) * bx
            probe_rows.append((a, a + 4 * bx))
    host = torch.empty(sum(b - a for a, b in probe_rows), dtype=torch.float64, pin_memory=True)
    d2h = host.numel() * 8
    e2e_time = 0.0
    for k in range(steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.selm_comp_sample(c, cycles_per_sample, xi)
        o = 0
        for a, b in probe_rows:
            host[o:o + b - a].copy_(xi[a:b], non_blocking=True)
            o += b - a
        torch.cuda.synchronize()
        e2e_time += time.perf_counter() - t0
    e2e_value = cells * cycles_per_sample * steps / e2e_time

    # per-kernel device time and the byte model of each class (one FAC cycle)
    prof_samples = min(steps, 3)
    S.selm_profile_reset()
    S.selm_profile_enable(True)
    for _ in range(prof_samples):
        S.selm_comp_sample(c, cycles_per_sample)
    torch.cuda.synchronize()
    S.selm_profile_enable(False)
    per_class = {}
    for ci, name in enumerate(S.KERNEL_CLASSES):
        ms, cnt = S.selm_profile_read(ci)
        per_class[name] = {"ms": ms, "launches": cnt}
    S.selm_profile_reset()
    ncyc = prof_samples * cycles_per_sample
    N0, N1 = 3 * fsize, 3 * bsize
    nu = 2
    late = 3 * 2 * fy * fx           # cells of the two interface layers
    ef = e / 4.0
    # section 8(d)'s fused model: 12 B per unknown-sweep (x e/4) on the level a
    # class sweeps; 65 B per unknown-cycle on the base levels below level 1;
    # FP64 refinement 20 B per unknown for the residual and 20 B for the update
    base_levels = N1 / 7.0            # levels 2.. of the base hierarchy: N1 (1/8 + 1/64 + ...)
    model = {   # algorithmic bytes per FAC cycle
        "fine_sweep": nu * MODEL_SWEEP_B * ef * N0,              # nu patch sweeps
        "coarse_sweep": 4 * MODEL_SWEEP_B * ef * N1 + MODEL_LEVEL_B * ef * base_levels,
        "outer_residual": 20.0 * (N0 + N1),
        "outer_update": 20.0 * (N0 + N1),
    }
    per_pass = {   # the kernels as built: every pass reads its whole level
        "fine_sweep": nu * (2 * e * (N0 + N0) + 2 * e * (late + late / 2)),
        "coarse_sweep": 4 * 2 * e * 2 * N1,
        "outer_residual": (16 + e) * (N0 + N1),
        "outer_update": (16 + e) * (N0 + N1),
    }
    tot_ms = sum(v["ms"] for v in per_class.values()) or 1.0
    peak, peak_kind = measured_peaks()
    rooflines = {}
    for name, b_cycle in model.items():
        pc = per_class[name]
        if pc["launches"] == 0:
            continue
        sec = pc["ms"] / 1e3
        achieved = b_cycle * ncyc / sec / 1e9
        rooflines[name] = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "peak_source": peak_kind, "traffic": None,
                           "algorithmic_bytes_per_launch": b_cycle * ncyc / pc["launches"],
                           "per_pass_model": {"bytes_per_launch": per_pass[name] * ncyc / pc["launches"],
                                              "frac": per_pass[name] * ncyc / sec / 1e9 / peak},
                           "avg_launch_us": pc["ms"] / pc["launches"] * 1e3,
                           "share_of_kernel_time": pc["ms"] / tot_ms}
    dominant = max(rooflines, key=lambda k: rooflines[k]["share_of_kernel_time"])
    roof = dict(rooflines[dominant])
    roof["others"] = {k: v for k, v in rooflines.items() if k != dominant}
    # a class mixes several kernels here, so the ncu traffic is given per kernel
    roof["ncu_traffic_per_launch_by_kernel"] = composite_ncu_traffic() or None
    unknown_cycles = (N0 + 3 * (bz - K) * by * bx) * cycles_per_sample
    roof["whole_step_model"] = {
        "bytes_per_step": MODEL_CYCLE_B * unknown_cycles,
        "frac": MODEL_CYCLE_B * unknown_cycles / (t_total / steps) / 1e9 / peak,
        "note": "114 B per unknown-cycle x composite unknowns x FAC cycles per sample / ms per sample"}

    # covariance of the probe block across the interface against the oracle's block
    cov = None
    exact = golden_block(n, K)
    if exact is not None and cov_samples > 0:
        from paper_1003_2680_gb300 import covariance as CV
        est, se, ns = CV.composite_block(c, n, K, 3, nsamples=cov_samples, nbatches=10)
        cov = dict(CV.compare(est, se, exact), samples=ns,
                   block="4^3 probe block of one component across the coarse-fine interface (x, y = 126..129 "
                         "in each level's indexing; fine layers 2K-2, 2K-1 and base rows K+1, K+2), averaged "
                         "over all x-y base-cell translates and the 3 components",
                   exact="A^-1 block from the oracle's composite FAC solves (tests/golden)")
    cpu = composite_cpu_baseline(128, 16) if with_cpu else None
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": 1e3 * t_total / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
        "config": {"workload": f"composite grid: {n}^3 channel (periodic x-y, walls z) with its bottom {K} rows "
                               f"refined by 2 (patch {fx}x{fy}x{fz}), 3 components, thermal samples of "
                               f"{cycles_per_sample} stochastic FAC cycles (Algorithms 1-2), FP32 inner cycles; "
                               f"chain residual and update in double-float (two FP32 words, ~48 bits), "
                               f"FP64 coarsest solve",
                   "base_n": n, "patch_rows": K, "cells": cells, "unknowns": N0 + 3 * (bz - K) * by * bx,
                   "l2": "flushed between samples (256 MB write, outside the timed events)",
                   "unit_of_work": "cell-cycle = one cell (base or patch, all 3 components) through one FAC cycle",
                   "parallelism": "replicas x1"},
        "kernel_time_share": {k: round(v["ms"] / tot_ms, 4) for k, v in per_class.items() if v["launches"]},
        "roofline": roof,
        "covariance": cov,
        "e2e": {"value": e2e_value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    S.selm_comp_destroy(c)
    return line


def mac_measure(S, n, K, steps, warmup, particles=1000):
    """The staggered composite grid with the projection (selm_mac.h): the
    {n}^3 MAC channel with its bottom K rows refined by 2, FP32 inner cycles
    with FP64 residual and update.  Timed: thermal samples of the chain (2
    stochastic FAC cycles each, Algorithms 1-2 on the composite velocity
    operator) and Euler-Maruyama steps of `particles` particles (Algorithm 4:
    spread, P~^T, FAC solve to 1e-10, 2 chain cycles, P~, interpolation)."""
    import numpy as np
    import torch
    import selm_inputs
    cycles_per_sample = SAMPLE_CYCLES
    t0 = time.perf_counter()
    h = S.selm_mac_create(S.make_mac_desc(3, n, K, kT=1.0, precision=S.SELM_FP32_REFINE64,
                                          projection=S.SELM_PROJ_MAC, seed=0, instance=0))
    setup_s = time.perf_counter() - t0
    nf, ncells = S.selm_mac_faces(h), S.selm_mac_cells(h)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(warmup):
        S.selm_mac_sample(h, cycles_per_sample)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    launches0 = S.selm_kernel_launches()
    print(f"[bench] library kernel launches before the timed region: {launches0}", file=sys.stderr)
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(steps):
            flush.fill_(float(k))
            ev[k][0].record()
            S.selm_mac_sample(h, cycles_per_sample)
            ev[k][1].record()
        torch.cuda.synchronize()
    launches = S.selm_kernel_launches() - launches0
    t_total = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    value = ncells * cycles_per_sample * steps / t_total
    # per-class device time of the chain cycles
    S.selm_profile_reset()
    S.selm_profile_enable(True)
    for _ in range(2):
        S.selm_mac_sample(h, cycles_per_sample)
    torch.cuda.synchronize()
    S.selm_profile_enable(False)
    per_class = {}
    for ci, name in enumerate(S.KERNEL_CLASSES):
        ms, cnt = S.selm_profile_read(ci)
        if cnt:
            per_class[name] = {"ms": ms, "launches": cnt}
    S.selm_profile_reset()
    tot_ms = sum(v["ms"] for v in per_class.values()) or 1.0
    # Euler-Maruyama steps with particles (projection on)
    X0 = selm_inputs.particles(particles, 3, 2 * n, seed=0)
    F0 = selm_inputs.forces(particles, 3, seed=0)
    X = torch.tensor(X0, device="cuda")
    F = torch.tensor(F0, device="cuda")
    S.selm_mac_step(h, X, F, 1e-3, 1, cycles_per_sample)
    torch.cuda.synchronize()
    c0 = S.selm_mac_total_cycles(h)
    em_steps = max(2, steps // 4)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    S.selm_mac_step(h, X, F, 1e-3, em_steps, cycles_per_sample)
    b.record()
    torch.cuda.synchronize()
    em_ms = a.elapsed_time(b) / em_steps
    em_cycles = (S.selm_mac_total_cycles(h) - c0) / em_steps
    u = torch.randn(nf, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    a.record()
    it, res = S.selm_mac_project(h, u, out)
    b.record()
    torch.cuda.synchronize()
    proj_ms = a.elapsed_time(b)
    peak, peak_kind = measured_peaks()
    whole = MODEL_CYCLE_B * nf * cycles_per_sample
    S.selm_mac_destroy(h)
    return {
        "value": value, "unit": "cells/s", "ms_per_step": 1e3 * t_total / steps, "steps": steps, "warmup": warmup,
        "dtype": "f32+f64",
        "config": {"workload": f"staggered composite MAC grid: {n}^3 channel (periodic x-y, walls z) with its "
                               f"bottom {K} rows refined by 2, thermal samples of {cycles_per_sample} stochastic "
                               f"FAC cycles (explicit sparse operators, first-fit colour classes), FP32 inner "
                               f"cycles, FP64 residual, update and coarsest draw",
                   "base_n": n, "patch_rows": K, "cells": ncells, "face_unknowns": nf,
                   "l2": "flushed between samples (256 MB write, outside the timed events)",
                   "unit_of_work": "cell-cycle = one composite cell (all face unknowns it owns) through one FAC cycle",
                   "host_setup_s": setup_s},
        "kernel_time_share": {k: round(v["ms"] / tot_ms, 4) for k, v in per_class.items()},
        "avg_launch_us": {k: 1e3 * v["ms"] / v["launches"] for k, v in per_class.items()},
        "whole_step_model": {"bytes_per_sample": whole, "frac": whole / (t_total / steps) / 1e9 / peak,
                             "peak": peak, "peak_source": peak_kind,
                             "note": "114 B per unknown-cycle x face unknowns x cycles per sample / ms per sample"},
        "em_step": {"particles": particles, "ms_per_step": em_ms, "fac_cycles_per_step": em_cycles,
                    "projections_per_step": 3},
        "projection": {"ms": proj_ms, "cg_iterations": it, "relative_residual": res},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }


def stokes_measure(S, n, particles, steps, warmup):
    """The exact-Stokes Euler-Maruyama step with the Ito drift (f3): the n^3
    channel, FP32 inner cycles with FP64 refinement, `particles` particles;
    each step = the random-finite-difference drift (two Stokes mobility
    solves), 2 chain cycles and one Stokes solve of the combined forced and
    thermal field.  Every Stokes solve is conjugate gradients on the pressure
    Schur complement with FAC inner solves."""
    import torch
    import selm_inputs
    d = S.make_desc(dim=3, n=n, kT=1.0, precision=S.SELM_FP32_REFINE64, seed=0, instance=0,
                    max_particles=particles, torch_allocator=False)
    h = S.selm_mg_create(d)
    X = torch.tensor(selm_inputs.particles(particles, 3, n, seed=0), device="cuda")
    F = torch.tensor(selm_inputs.forces(particles, 3, seed=0), device="cuda")
    for _ in range(warmup):
        S.selm_mg_stokes_step(h, X, F, DT, 1, SAMPLE_CYCLES, 1e-4)
    torch.cuda.synchronize()
    c0 = S.selm_mg_stats(h)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = S.selm_kernel_launches()
    a.record()
    S.selm_mg_stokes_step(h, X, F, DT, steps, SAMPLE_CYCLES, 1e-4)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    launches = S.selm_kernel_launches() - launches0
    vcycles = (S.selm_mg_stats(h)[2] - c0[2]) / steps
    # one Stokes solve alone: outer iterations
    f = torch.randn(S.selm_mg_layout(h, S.SELM_SYS_VELOCITY, 0, 0)[2], dtype=torch.float64, device="cuda")
    u = torch.empty_like(f)
    it, res = S.selm_mg_stokes_solve(h, f, u)
    S.selm_mg_destroy(h)
    return {"workload": f"3-D {n}^3 channel, {particles} particles, exact Stokes mobility + Ito drift "
                        f"(random finite difference, delta = 1e-4), 2 chain cycles per step, FP32 inner cycles with "
                        f"FP64 refinement",
            "ms_per_step": ms, "vcycles_per_step": vcycles, "stokes_solves_per_step": 3,
            "cell_cycles_per_s": n ** 3 * vcycles / (ms / 1e3),
            "schur_cg_iterations_per_solve": it, "schur_relative_residual": res,
            "gpu_launches_per_step": launches / steps}


def run_mac(args):
    from paper_1003_2680_gb300 import _build
    _build.build()
    from paper_1003_2680_gb300 import selm as S
    line = mac_measure(S, args.mac_n, args.mac_k, args.steps, args.warmup)
    line.update({"metric": METRIC, "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                 "data": "synthetic", "cpu_baseline": None})
    print(json.dumps(line), flush=True)


def run_composite(args):
    """Composite grid: 256^3 base channel with its bottom 32 rows refined by 2
    (patch 512 x 512 x 64), three components, thermal samples of the chain
    (2 stochastic composite FAC cycles per sample)."""
    from paper_1003_2680_gb300 import _build
    _build.build()
    from paper_1003_2680_gb300 import selm as S
    line = composite_measure(S, args.comp_n, args.comp_k, args.steps, args.warmup, not args.no_cpu_baseline,
                             cov_samples=200)
    print(json.dumps(line), flush=True)


def config1_measure(S):
    """The 64^2 2-D plain method in FP64 (6 levels, (2,2) sweeps, Cholesky
    coarsest, Philox seed 0, 16 particles): 1000 stochastic cycles of the
    chain and the 32 x 32 mobility (32 unit-force solves), as latencies."""
    import numpy as np
    import torch
    import selm_inputs
    m = S.SelmMG(dim=2, n=64, levels=6, precision=S.SELM_FP64, seed=0, instance=0)
    X = torch.tensor(selm_inputs.particles(16, 2, 64, seed=0), device="cuda")
    g = torch.zeros_like(X)
    S.selm_mg_sample(m.h, X, 20, g)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    S.selm_mg_sample(m.h, X, 1000, g)
    b.record()
    torch.cuda.synchronize()
    t_chain = a.elapsed_time(b) / 1e3
    U = torch.zeros_like(X)
    cols, solve_cycles = [], 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for col in range(32):
        F = torch.zeros_like(X)
        F[col // 2, col % 2] = 1.0
        cyc, _ = S.selm_mg_solve(m.h, X, F, U)
        solve_cycles += cyc
        cols.append(U.clone())
    torch.cuda.synchronize()
    t_mob = time.perf_counter() - t0
    M = torch.stack(cols, dim=2).reshape(32, 32).cpu().numpy()
    m.close()
    return {"workload": "2-D 64^2 plain method, FP64, 6 levels, (2,2) red-black sweeps, Cholesky coarsest",
            "chain_us_per_cycle": 1e6 * t_chain / 1000,
            "mobility_32x32_ms": 1e3 * t_mob, "mobility_fac_cycles": solve_cycles,
            "mobility_symmetry": float(np.abs(M - M.T).max() / np.abs(M).max()),
            "mobility_min_eig": float(np.linalg.eigvalsh(0.5 * (M + M.T)).min())}


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    assert args.warmup >= 3, "at least 3 warm-up steps"
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "served":
        run_served(args)
        return
    if args.workload == "mac":
        return run_mac(args)
    if args.workload == "composite":
        run_composite(args)
        return
    if args.workload == "decorrelation":
        run_decorrelation(args)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1003_2680_gb300 import _build
    _build.build()
    from paper_1003_2680_gb300 import selm as S
    import selm_inputs

    n, npart = args.n, args.particles
    proj = S.SELM_PROJ_NONE if args.no_projection else S.SELM_PROJ_MAC
    m = S.SelmMG(dim=3, n=n, precision=S.SELM_FP32_REFINE64, projection=proj, tol=1e-10, seed=0,
                 instance=rank, max_particles=npart)
    h = m.h
    if args.engine_level:
        S.selm_mg_set_option(h, S.SELM_OPT_ENGINE_LEVEL, args.engine_level)
    X0 = selm_inputs.particles(npart, 3, n, seed=rank)
    F0 = selm_inputs.forces(npart, 3, seed=rank)
    X = torch.tensor(X0, device="cuda")
    F = torch.tensor(F0, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    pres_steps = [0]
    spectral = S.selm_mg_pressure_spectral(h) == 1 if proj == S.SELM_PROJ_MAC else False

    def one_step():
        S.selm_mg_step(h, X, F, DT, 1, SAMPLE_CYCLES)
        st = S.selm_mg_stats(h)
        pres_steps[0] += st[1]   # pressure V-cycles, or spectral refinement iterations
        return st[0] + SAMPLE_CYCLES

    # burn-in of the chain + warm-up of every path
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # ---- timed region (device events per step, L2 flushed between steps) ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    cycles = 0
    pres_before = pres_steps[0]
    launches0 = S.selm_kernel_launches()
    print(f"[bench] library kernel launches before the timed region: {launches0}", file=sys.stderr)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            cycles += one_step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = S.selm_kernel_launches() - launches0
    pres_steps_cycles = pres_steps[0] - pres_before
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = sum(step_ms) / 1e3
    t_total, cycles_all = whole_job(t_total, cycles, world, "cuda")
    value = n ** 3 * cycles_all / t_total

    # ---- end to end: the host-buffer C call, copies inside the timed region ----
    Xh = torch.tensor(X0).pin_memory()
    Fh = torch.tensor(F0).pin_memory()
    for _ in range(2):
        S.selm_mg_step_host(h, Xh, Fh, DT, 1, SAMPLE_CYCLES)
    e2e_time, e2e_cycles = 0.0, 0
    torch.cuda.synchronize()
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.selm_mg_step_host(h, Xh, Fh, DT, 1, SAMPLE_CYCLES)
        e2e_time += time.perf_counter() - t0
        e2e_cycles += S.selm_mg_stats(h)[0] + SAMPLE_CYCLES
    barrier()
    e2e_time, e2e_units = whole_job(e2e_time, e2e_cycles, world, "cuda")
    e2e_value = n ** 3 * e2e_units / e2e_time

    # ---- per-kernel device time (events on the launching stream) ----
    prof_steps = min(args.steps, 3)
    S.selm_profile_reset()
    S.selm_profile_enable(True)
    vel_cycles = pres_cycles = 0
    for _ in range(prof_steps):
        one_step()
        st = S.selm_mg_stats(h)
        vel_cycles += st[0] + SAMPLE_CYCLES
        pres_cycles += st[1]
    torch.cuda.synchronize()
    S.selm_profile_enable(False)
    per_class = {}
    for ci, name in enumerate(S.KERNEL_CLASSES):
        ms, cnt = S.selm_profile_read(ci)
        per_class[name] = {"ms": ms, "launches": cnt}
    S.selm_profile_reset()
    tot_ms = sum(v["ms"] for v in per_class.values()) or 1.0
    dominant = max(per_class, key=lambda k: per_class[k]["ms"])
    peak, peak_kind = measured_peaks()
    # section 8(d)'s byte model (the roofline's algorithmic bytes) and, as a
    # labelled extra, the per-colour-pass bytes of the kernels as built
    coarse_model = vel_cycles * model_coarse_bytes_per_vcycle(S, h, 0)
    coarse_pass = vel_cycles * coarse_bytes_per_vcycle(S, h, 0)
    if proj == S.SELM_PROJ_MAC:
        coarse_model += pres_cycles * model_coarse_bytes_per_vcycle(S, h, 1)
        coarse_pass += pres_cycles * coarse_bytes_per_vcycle(S, h, 1)
    roof = None
    for name in (dominant, "fine_sweep"):
        if name not in ("fine_sweep", "coarse_sweep") or per_class[name]["launches"] == 0:
            continue
        nl = per_class[name]["launches"]
        avg_s = per_class[name]["ms"] / nl / 1e3
        if name == "fine_sweep":
            bytes_launch = model_fine_bytes_per_colour_launch(S, h)
            pass_launch = fine_bytes_per_launch(S, h)
        else:   # engine and cooperative launches: the coarse bytes of the profiled steps over their launches
            bytes_launch = coarse_model / nl
            pass_launch = coarse_pass / nl
        achieved = bytes_launch / avg_s / 1e9
        entry = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                 "frac": achieved / peak, "peak_source": peak_kind,
                 "traffic": ncu_traffic(name, n), "algorithmic_bytes_per_launch": bytes_launch,
                 "bytes_model": "section 8(d): 12 B per unknown-sweep (fused red+black) on the finest level; "
                                "65 B per unknown-cycle on each coarse level",
                 "per_pass_model": {"bytes_per_launch": pass_launch,
                                    "achieved": pass_launch / avg_s / 1e9,
                                    "frac": pass_launch / avg_s / 1e9 / peak,
                                    "note": "every colour pass reads its whole level, reads b and writes v "
                                            "at its colour (the kernels as built)"},
                 "avg_launch_us": avg_s * 1e6, "share_of_kernel_time": per_class[name]["ms"] / tot_ms}
        if roof is None:
            roof = entry
        else:
            roof["fine_sweep"] = entry
    if roof is None:
        roof = {"bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None, "traffic": None}
    # whole step against the 114 B per unknown-cycle model, over every V-cycle
    # executed (velocity solve + chain, and the projections' pressure solves)
    n_vel = level_unknowns(S, h, 0)[0]
    n_pres = level_unknowns(S, h, 1)[0] if proj == S.SELM_PROJ_MAC else 0
    vel_per_step = cycles_all / args.steps / world
    pres_iter_per_step = pres_steps_cycles / args.steps if args.steps else 0.0
    pres_per_step = 0.0 if spectral else pres_iter_per_step   # pressure V-cycles
    unknown_cycles_step = vel_per_step * n_vel + pres_per_step * n_pres
    step_s = t_total / args.steps
    roof["whole_step_model"] = {
        "bytes_per_step": MODEL_CYCLE_B * unknown_cycles_step,
        "achieved": MODEL_CYCLE_B * unknown_cycles_step / step_s / 1e9,
        "frac": MODEL_CYCLE_B * unknown_cycles_step / step_s / 1e9 / peak,
        "note": "114 B per unknown-cycle x every V-cycle of the step (velocity and pressure) / ms_per_step"}

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(workload_config(n, npart, proj == S.SELM_PROJ_MAC), levels=S.selm_mg_levels(h, 0),
                       engine_first_level=S.selm_mg_engine_info(h)[0],
                       parallelism=f"replicas x{world} (independent systems, no collective on the data path)"),
        "velocity_vcycles_per_step": cycles_all / args.steps / world,
        "vcycles_per_step": {"velocity": vel_per_step, "pressure": pres_per_step,
                             "total": vel_per_step + pres_per_step},
        "pressure_solve": ({"inner": "spectral (FFT along x, y; tridiagonal along z; FP32) in FP64 refinement",
                            "refinement_iterations_per_step": pres_iter_per_step} if spectral else
                           {"inner": "V-cycle of the pressure system in FP64 refinement",
                            "vcycles_per_step": pres_iter_per_step}),
        "unknown_cycles_per_s_all_vcycles": unknown_cycles_step / step_s * world,
        "roofline": roof,
        "kernel_time_share": {k: round(v["ms"] / tot_ms, 4) for k, v in per_class.items() if v["launches"]},
        "e2e": {"value": e2e_value, "unit": "cells/s",
                "h2d_bytes_per_step": int(X0.nbytes + F0.nbytes), "d2h_bytes_per_step": int(X0.nbytes)},
        "gpu_launches": int(launches),
        "clocks": {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
    }
    # the same step with the projection's pressure solved by V-cycles (the
    # multigrid path the composite grid uses), timed the same way
    if spectral and not args.no_extras:
        S.selm_mg_set_option(h, S.SELM_OPT_PRESSURE_SPECTRAL, 0)
        for _ in range(2):
            one_step()
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        cyc2, p0 = 0, pres_steps[0]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev2[k][0].record(stream)
            cyc2 += one_step()
            ev2[k][1].record(stream)
        torch.cuda.synchronize()
        t2 = sum(a.elapsed_time(b) for a, b in ev2) / 1e3
        pv = (pres_steps[0] - p0) / args.steps
        line["mg_projection"] = {
            "value": n ** 3 * cyc2 / t2, "unit": "cells/s", "ms_per_step": 1e3 * t2 / args.steps,
            "vcycles_per_step": {"velocity": cyc2 / args.steps, "pressure": pv, "total": cyc2 / args.steps + pv},
            "unknown_cycles_per_s_all_vcycles": (cyc2 / args.steps * n_vel + pv * n_pres) / (t2 / args.steps),
            "note": "the same workload with the projection's pressure solved by V-cycles of the pressure system"}
        S.selm_mg_set_option(h, S.SELM_OPT_PRESSURE_SPECTRAL, 1)
    # the chain's sample covariance on 4^3 wall blocks of every velocity
    # component against the exact A^-1 blocks (spectral closed form)
    if not args.no_extras:
        line["covariance"] = channel_covariance(S, h, n)
    m.close()
    if rank == 0 and not args.no_extras:
        # the composite workload (the HBM-bound configuration) and the 2-D
        # 64^2 FP64 configuration, measured in the same run
        torch.cuda.empty_cache()
        comp = composite_measure(S, args.comp_n, args.comp_k, steps=60, warmup=3, with_cpu=False)
        line["composite"] = {k: comp[k] for k in ("value", "unit", "ms_per_step", "dtype", "config", "roofline",
                                                  "covariance", "e2e", "gpu_launches", "clocks",
                                                  "kernel_time_share", "steps", "warmup")}
        line["config1_64x64_fp64"] = config1_measure(S)
        torch.cuda.empty_cache()
        mac = mac_measure(S, 64, 8, steps=20, warmup=3)
        line["staggered_composite"] = {k: mac[k] for k in ("value", "unit", "ms_per_step", "dtype", "config",
                                                          "kernel_time_share", "avg_launch_us", "whole_step_model",
                                                          "em_step", "projection", "gpu_launches", "clocks")}
        line["stokes_drift_64"] = stokes_measure(S, 64, 256, steps=3, warmup=3)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(n)
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
