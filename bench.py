"""Benchmark: D3Q19 GLUPS and fraction of the HBM roofline on one GB300.

Default workload (the lid-driven cavity the metric is quoted on): dense
256^3 D3Q19, FP32 storage, BGK tau = 0.515, regularized lid u = 0.05 on the
top plane, bounce-back on the other walls, disaggregated schedule (lean
interior kernel + regularized lid kernel).  One bench step = one lattice
time step over the whole grid.  The 2.55 GB population state is ~20x the
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Every result carries its velocity-L2 error against
the FP64 oracle ("velocity_l2_vs_fp64"): the line's kernels run a reduced
case of the same workload whose oracle velocities are stored in
tests/golden/ (written by oracle/make_bench_references.py; the bench itself
runs no oracle code for this).  cpu_baseline times the FP64 oracle on the
host cores (one single-threaded process per core, and one alone);
--impl reference times the same oracle as the reference arm.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

if "--cpu-sample" in sys.argv:
    # a CPU-baseline child: one thread per process (the parent also sets these)
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = {"f32": 152, "f16": 76, "bf16": 76}   # 19 loads + 19 stores
NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e nominal bandwidth (context beside the measured copy peak)
METRIC = "D3Q19 GLUPS & % HBM roofline, FP32 vs FP16-store/learned at stated error"

# DRAM traffic of the dominant kernel from an ncu capture (profiles/), valid
# only while the kernel sources hash to the recorded value: the 160^3
# capture of dense_interior (dram__bytes_read.sum + dram__bytes_write.sum,
# 4,070,400 updates per launch) scaled by units to one 256^3 launch
# (16,711,680 updates), profiles/dense_interior_cavity160_ncu.md; keyed by
# kernel and storage (the FP16 capture: dense_interior_f16_cavity160_ncu.md).
NCU_TRAFFIC = {("dense_interior", "f32"): {"bytes_per_launch": 2.342294e+09, "src_sha": "27e849b9f3a71c23"},
               ("dense_interior", "f16"): {"bytes_per_launch": 1.109482e+09, "src_sha": "27e849b9f3a71c23"}}


def src_hash():
    h = hashlib.sha256()
    for f in ("d3q19.cuh", "dense.cuh", "dense.cu"):
        h.update(open(os.path.join(ROOT, "paper_2503_07898_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return None
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[3 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ------------------------------------------------------------------ oracle

def cpu_sample(n, steps, warmup):
    """Child process body: the FP64 oracle as it stands on an n^3 cavity (the
    GPU workload's boundaries, tau 0.515, lid 0.05); prints its timed window."""
    from oracle import lbm as olbm
    from paper_2503_07898_gb300 import workloads as wl
    flags, bc = wl.cavity(n, u_lid=0.05)
    f = olbm.init_equilibrium(np.ones((n, n, n)), np.zeros((3, n, n, n)))
    for _ in range(warmup):
        f = olbm.step(f, flags, 0.515, bc=bc)
    t0 = time.time()
    for _ in range(steps):
        f = olbm.step(f, flags, 0.515, bc=bc)
    t1 = time.time()
    print(json.dumps({"updates": n ** 3 * steps, "t0": t0, "t1": t1}), flush=True)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_cpu_glups(n, steps, warmup, procs):
    """GLUPS of `procs` single-threaded oracle processes running the n^3
    cavity sample side by side: all their updates over the span from the
    first timed window's start to the last one's end (the processes start
    together; interpreter start-up and warm-up lie outside the windows).
    Returns (GLUPS, seconds)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", str(n), str(steps),
           str(warmup)]
    ps = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                           env=env) for _ in range(procs)]
    rows = []
    for p in ps:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("CPU baseline sample failed")
        rows.append(json.loads(out.strip().splitlines()[-1]))
    span = max(r["t1"] for r in rows) - min(r["t0"] for r in rows)
    return sum(r["updates"] for r in rows) / span / 1e9, span


def cpu_baseline_line(n=64, steps=100):
    """The oracle timed on the host cores: one single-threaded process, then
    one per available core side by side (about 20 s of host time)."""
    cores = host_cores()
    one, dt1 = oracle_cpu_glups(n, steps, 1, 1)
    allc, dta = oracle_cpu_glups(n, steps, 1, cores)
    return {"value": allc, "unit": "GLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{n}^3 cavity (tau 0.515, lid 0.05), {steps} steps per process, numpy FP64, "
                      f"one thread per process ({cores} processes side by side, {dta:.1f} s)",
            "single_core": {"value": one, "unit": "GLUPS", "cores": 1, "seconds": round(dt1, 2)},
            "nproc": os.cpu_count(), "threads_per_process": 1}


def max_over_ranks(dist, x, device):
    """The largest per-rank float over all ranks (the job ends with its
    slowest replica); x itself without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_glups(world, updates_per_rank, steps, seconds):
    """Whole-job GLUPS of `world` independent replicas (weak scaling): the
    updates of every rank over the slowest rank's time."""
    return world * updates_per_rank * steps / seconds / 1e9


def run_reference(args, rank, world):
    if rank != 0:
        return
    n = 48 if args.steps <= 1000 else 32
    cores = host_cores()
    value, dt = oracle_cpu_glups(n, args.steps, args.warmup, cores)
    sample = (f"{n}^3 cavity window of the 256^3 workload per process (tau 0.515, lid 0.05), "
              f"numpy FP64, one thread per process, {cores} processes side by side")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cavity256 (sampled)", "sample": sample},
            "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- GPU

def _time_steps(torch, lbm, step, stream, n):
    """Device time of n calls of step() on stream, in ms."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(n)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


REFS = os.path.join(ROOT, "tests", "golden", "bench_velocity_references.npz")


class Accuracy:
    """Velocity-L2 error against the FP64 oracle of a bench line's form: the
    reduced case of the line's workload (workloads.accuracy_cases: same
    layout, boundaries, relaxation time and start, small enough for the
    oracle) runs through the library with the line's storage, collision,
    schedule and kernel variant; its velocity at the case's sampled updated
    voxels is compared with the oracle's, stored by
    oracle/make_bench_references.py (the bench never runs the oracle for
    this).  L2 = sqrt(sum |u - u_ref|^2 / sum |u_ref|^2) over the samples,
    each sample weighted by the volume it stands for (8^l times the level's
    updated voxels over its samples on multi-resolution grids)."""

    def __init__(self, lbm, wl):
        self.lbm, self.wl = lbm, wl
        self.cases = wl.accuracy_cases()
        self.refs = dict(np.load(REFS)) if os.path.exists(REFS) else {}
        self.manifest = json.loads(str(self.refs["manifest"])) if "manifest" in self.refs else {}

    def _bc_list(self, flags, bc):
        t = flags & 7
        return np.ascontiguousarray(bc[:, (t == 2) | (t == 3)].T, np.float32)

    def _gpu(self, case, samples, storage, collision, schedule, variant, theta):
        """Velocities at the samples after the case's steps, and the weight of
        each sample set."""
        lbm, wl = self.lbm, self.wl
        kind = case["kind"]
        if kind in ("dense", "sparse"):
            flags = case["flags"]
            nz, ny, nx = flags.shape
            phys = lbm.physics(case["tau"], collision, storage, case["periodic"], schedule,
                               lattice=case["q"])
            if kind == "dense":
                g = lbm.lbm_grid_create_dense((nx, ny, nz), phys)
                lbm.lbm_set_boundary(g, 0, flags, self._bc_list(flags, case["bc"]))
            else:
                g = lbm.lbm_grid_create_sparse((nx, ny, nz), 8, flags, phys)
                lbm.lbm_set_boundary(g, 0, None, self._bc_list(flags, case["bc"]))
            if variant is not None:
                lbm.lbm_set_variant(g, variant)
            rho, u = case["fields"][0]
            lbm.lbm_init_equilibrium(g, 0, rho, u)
            lbm.lbm_step(g, case["steps"])
            _, ug = lbm.lbm_get_moments(g, 0)
            lbm.lbm_grid_destroy(g)
            return [ug.reshape(3, -1)[:, samples[0]]], [1.0]
        if kind == "batch":
            grids = []
            for c in case["cases"]:
                phys = lbm.physics(c["tau"], collision, storage, (1, 1, 1))
                if c["kind"] == "dense":
                    g = lbm.lbm_grid_create_dense(c["dims"], phys)
                    lbm.lbm_set_boundary(g, 0, c["flags"])
                else:
                    g = lbm.lbm_grid_create_sparse(c["dims"], 8, c["flags"], phys)
                lbm.lbm_init_equilibrium(g, 0, *wl.batch_case_fields(c))
                grids.append(g)
            b = lbm.lbm_batch_create(grids)
            if theta is not None:
                lbm.lbm_batch_closure_load(b, theta, 64)
            lbm.lbm_batch_step(b, case["steps"])
            us, ws = [], []
            for g, idx in zip(grids, samples):
                us.append(lbm.lbm_get_moments(g, 0)[1].reshape(3, -1)[:, idx])
                ws.append(lbm.lbm_get_info(g)["n_updated"][0] / len(idx))
            del b
            for g in grids:
                lbm.lbm_grid_destroy(g)
            return us, ws
        L = case["n_levels"]
        phys = lbm.physics(case["tau"], collision, storage, case["periodic"], schedule,
                           closure=1 if theta is not None else 0, lattice=case["q"])
        g = lbm.lbm_grid_create_multires(case["dims"], L, case["level_map"], phys)
        if variant is not None:
            lbm.lbm_set_variant(g, variant)
        if case["flags"] is not None:
            lbm.lbm_set_boundary(g, 0, case["flags"], self._bc_list(case["flags"], case["bc"]))
        if theta is not None:
            lbm.lbm_closure_load(g, theta)
        for lv, (rho, u) in enumerate(case["fields"]):
            lbm.lbm_init_equilibrium(g, lv, rho, u)
        lbm.lbm_step(g, case["steps"])
        info = lbm.lbm_get_info(g)
        us = [lbm.lbm_get_moments(g, lv)[1].reshape(3, -1)[:, samples[lv]] for lv in range(L)]
        ws = [8.0 ** lv * info["n_updated"][lv] / max(1, len(samples[lv])) for lv in range(L)]
        lbm.lbm_grid_destroy(g)
        return us, ws

    def run(self, name, storage="f32", collision="bgk", schedule="disaggregated", variant=None):
        case = self.cases[name]
        samples = self.wl.accuracy_samples(case)
        steps_key = "after_coarsest_steps" if case["kind"] == "multires" else "after_steps"
        base = {"l2_case": name, steps_key: case["steps"]}
        for k, idx in enumerate(samples):
            ref = self.refs.get(f"{name}/idx{k}")
            if ref is None or not np.array_equal(ref, idx):
                return dict(base, velocity_l2_vs_fp64=None, why="no stored oracle reference")
        us, ws = self._gpu(case, samples, storage, collision, schedule, variant,
                           case.get("theta"))
        num = den = 0.0
        for k, (u, w) in enumerate(zip(us, ws)):
            ur = self.refs[f"{name}/u{k}"].astype(np.float64)
            num += w * float(((u - ur) ** 2).sum())
            den += w * float((ur ** 2).sum())
        return dict(base, velocity_l2_vs_fp64=float(f"{np.sqrt(num / den):.3e}"))

    def cases_used(self):
        return {k: v["what"] for k, v in self.manifest.items()}


def measure_workloads(torch, lbm, wl, stream, peak, steps, which, acc, theta=None, n_batch=128):
    """GLUPS of the other layouts of the method on their full-size inputs
    (context lines of the same metric; each timed after 3 warm-up steps),
    each with its velocity-L2 error against the FP64 oracle (Accuracy).
    theta: the learned closure's trained weights for the closure lines
    (None: a fixed test network of the same size; the cost of inference does
    not depend on the values)."""
    STAGED = lbm.LBM_VARIANT_STAGED
    out = {}
    trained = theta is not None
    if theta is None:
        theta = wl.closure_test_network()
    if "sparse" in which:
        flags, bc = wl.sphere_channel()
        t = flags & 7
        bcl = np.ascontiguousarray(bc[:, (t == 2) | (t == 3)].T, np.float32)
        for key, q, cases in (
                ("sphere_channel_512x256x256_sparse8", 19,
                 (("disaggregated_f32", dict(storage="f32")),
                  ("disaggregated_f32_staged", dict(storage="f32", variant=STAGED)),
                  ("disaggregated_bitmask_f32", dict(storage="f32", schedule="bitmask")),
                  ("monolithic_f32", dict(storage="f32", schedule="monolithic")),
                  ("disaggregated_f16", dict(storage="f16")),
                  ("disaggregated_f16_staged", dict(storage="f16", variant=STAGED)))),
                # the paper's register-pressure configuration: D3Q27,
                # block-sparse, regularized inflow / outflow (Sec. 6.2)
                ("sphere_channel_512x256x256_sparse8_d3q27", 27,
                 (("disaggregated_f32", dict(storage="f32")),
                  ("disaggregated_f32_staged", dict(storage="f32", variant=STAGED)),
                  ("disaggregated_bitmask_f32", dict(storage="f32", schedule="bitmask")),
                  ("monolithic_f32", dict(storage="f32", schedule="monolithic"))))):
            res = {}
            for name, kw in cases:
                pk = {k: v for k, v in kw.items() if k != "variant"}
                g = lbm.lbm_grid_create_sparse(flags.shape[::-1], 8, flags,
                                               lbm.physics(0.52, lattice=q, **pk), stream=stream)
                if "variant" in kw:
                    lbm.lbm_set_variant(g, kw["variant"])
                lbm.lbm_set_boundary(g, 0, None, bcl)
                lbm.lbm_init_equilibrium(g, 0, None, None)
                n_upd = lbm.lbm_get_info(g)["n_updated"][0]
                lbm.lbm_step(g, 3, stream)
                ms = _time_steps(torch, lbm, lambda n: lbm.lbm_step(g, n, stream), stream, steps)
                bpu = 2 * q * (4 if kw["storage"] == "f32" else 2)
                glups = n_upd * steps / (ms * 1e-3) / 1e9
                res[name] = {"GLUPS": round(glups, 3),
                             "roofline_frac": round(glups * bpu / peak, 4),
                             "bytes_per_update": bpu}
                lbm.lbm_grid_destroy(g)
                res[name].update(acc.run(f"sphere_small_q{q}", storage=kw["storage"],
                                         schedule=kw.get("schedule", "disaggregated"),
                                         variant=kw.get("variant")))
            out[key] = res
    if "multires" in which or "turbulence" in which:
        # the configuration's start: seeded k^-5/3 field, u_rms 0.03, on the
        # 256^3 finest box, coarser levels the means over their cubes
        lmap = wl.multires_slab_map()
        rho, u = wl.turbulence(256, seed=7898, u_rms=0.03)
        fields = wl.level_fields(rho, u, 3)
        del rho, u
        res = {}
        for name, kw in (("fused_f32", dict()), ("fused_f32_staged", dict(variant=STAGED)),
                         ("unfused_f32", dict(schedule="monolithic")),
                         ("fused_f16", dict(storage="f16")),
                         ("fused_f16_staged", dict(storage="f16", variant=STAGED)),
                         ("fused_f32_learned_closure", dict(closure=1)),
                         ("fused_f32_d3q27", dict(lattice=27))):
            pk = {k: v for k, v in kw.items() if k != "variant"}
            g = lbm.lbm_grid_create_multires((256, 256, 256), 3, lmap,
                                             lbm.physics(0.52, periodic=(1, 1, 1), **pk),
                                             stream=stream)
            if "variant" in kw:
                lbm.lbm_set_variant(g, kw["variant"])
            if kw.get("closure"):
                lbm.lbm_closure_load(g, theta)
            info = lbm.lbm_get_info(g)
            ups = sum(n * 2 ** (2 - l) for l, n in enumerate(info["n_updated"]))
            for l in range(3):
                lbm.lbm_init_equilibrium(g, l, *fields[l])
            lbm.lbm_step(g, 3, stream)
            ms = _time_steps(torch, lbm, lambda n: lbm.lbm_step(g, n, stream), stream,
                             max(1, steps // 4))
            glups = ups * max(1, steps // 4) / (ms * 1e-3) / 1e9
            bpu = (76 if kw.get("storage") == "f16" else 152) * kw.get("lattice", 19) // 19
            res[name] = {"GLUPS": round(glups, 3), "roofline_frac": round(glups * bpu / peak, 4)}
            lbm.lbm_grid_destroy(g)
            acc_case = ("turb3_closure" if kw.get("closure") else
                        f"turb3_q{kw.get('lattice', 19)}")
            res[name].update(acc.run(acc_case, storage=kw.get("storage", "f32"),
                                     schedule=kw.get("schedule", "disaggregated"),
                                     variant=kw.get("variant")))
        res["updates_per_coarsest_step"] = ups
        res["start"] = "seeded k^-5/3 field (seed 7898, u_rms 0.03), coarse levels its cube means"
        res["closure_weights"] = ("trained (learned_closure_quality)" if trained else
                                  "a fixed test network (workloads.closure_test_network)")
        out["turbulence_256_3level"] = res
        del fields
    cavities = ((384, 3, (2, 2), "cavity3_160",
                 (("fused_f32", dict()), ("fused_f32_staged", dict(variant=STAGED)),
                  ("unfused_f32", dict(schedule="monolithic")),
                  ("fused_f16", dict(storage="f16")))),
                (512, 4, (1, 1, 1), "mr4_small",
                 (("fused_f32", dict()),
                  ("unfused_f32", dict(schedule="monolithic")))))
    for n, nlev, shells, acc_case, cases in (cavities if ("multires" in which or "cavity" in which)
                                             else ()):
        # the paper's multi-resolution benchmark (Sec. 6.3, Table 5): a
        # lid-driven cavity, finest level along the walls and the lid
        lmap = wl.multires_cavity_map(n, nlev, shells)
        flags, bc = wl.cavity(n)
        t = flags & 7
        bcl = np.ascontiguousarray(bc[:, (t == 2) | (t == 3)].T, np.float32)
        res = {}
        for name, kw in cases:
            pk = {k: v for k, v in kw.items() if k != "variant"}
            g = lbm.lbm_grid_create_multires((n,) * 3, nlev, lmap, lbm.physics(0.52, **pk),
                                             stream=stream)
            if "variant" in kw:
                lbm.lbm_set_variant(g, kw["variant"])
            lbm.lbm_set_boundary(g, 0, flags, bcl)
            info = lbm.lbm_get_info(g)
            ups = sum(k * 2 ** (nlev - 1 - l) for l, k in enumerate(info["n_updated"][:nlev]))
            for l in range(nlev):
                lbm.lbm_init_equilibrium(g, l, None, None)
            lbm.lbm_step(g, 3, stream)
            nst = max(1, steps // 4)
            ms = _time_steps(torch, lbm, lambda k: lbm.lbm_step(g, k, stream), stream, nst)
            glups = ups * nst / (ms * 1e-3) / 1e9
            bpu = 76 if kw.get("storage") == "f16" else 152
            res[name] = {"GLUPS": round(glups, 3), "roofline_frac": round(glups * bpu / peak, 4)}
            lbm.lbm_grid_destroy(g)
            res[name].update(acc.run(acc_case, storage=kw.get("storage", "f32"),
                                     schedule=kw.get("schedule", "disaggregated"),
                                     variant=kw.get("variant")))
        tot = n ** 3
        res["pct_of_finest_box_voxels"] = [round(100 * k / tot, 3) for k in info["n_updated"][:nlev]]
        res["voxels_per_level"] = list(info["n_updated"][:nlev])
        res["updates_per_coarsest_step"] = ups
        out[f"cavity_{n}_{nlev}level"] = res
    if "batch" in which:
        cases = wl.batch_cases(n_cases=n_batch)
        grids = []
        for c in cases:
            phys = lbm.physics(c["tau"], storage="f16", periodic=(1, 1, 1))
            if c["kind"] == "dense":
                g = lbm.lbm_grid_create_dense(c["dims"], phys, stream=stream)
                lbm.lbm_set_boundary(g, 0, c["flags"])
            else:
                g = lbm.lbm_grid_create_sparse(c["dims"], 8, c["flags"], phys, stream=stream)
            rho, u = wl.batch_case_fields(c)
            lbm.lbm_init_equilibrium(g, 0, rho, u)
            grids.append(g)
        b = lbm.lbm_batch_create(grids)
        k, _ = lbm.lbm_batch_autotune(b, 4)
        info = lbm.lbm_batch_info(b)
        lbm.lbm_batch_step(b, steps, stream)        # captures the graph
        torch.cuda.synchronize()
        ms = _time_steps(torch, lbm, lambda n: lbm.lbm_batch_step(b, n, stream), stream, steps)
        glups = info["n_updated"] * steps / (ms * 1e-3) / 1e9
        out[f"serving_batch_{n_batch}_f16"] = dict(
            {"GLUPS": round(glups, 3), "roofline_frac": round(glups * 76 / peak, 4),
             "updated_voxels": info["n_updated"], "ctas_per_sm": k, "launches_per_step": 1},
            **acc.run("batch_small", storage="f16"))
        # the learned closure on the cases whose largest edge is <= 64
        lbm.lbm_batch_closure_load(b, theta, 64)
        n_cl = sum(1 for c in cases if max(c["dims"]) <= 64)
        k, _ = lbm.lbm_batch_autotune(b, 4)
        lbm.lbm_batch_step(b, steps, stream)
        torch.cuda.synchronize()
        ms = _time_steps(torch, lbm, lambda n: lbm.lbm_batch_step(b, n, stream), stream, steps)
        glups = info["n_updated"] * steps / (ms * 1e-3) / 1e9
        out[f"serving_batch_{n_batch}_f16_learned_closure"] = dict(
            {"GLUPS": round(glups, 3), "roofline_frac": round(glups * 76 / peak, 4),
             "closure_cases": n_cl, "max_edge": 64, "ctas_per_sm": k, "launches_per_step": 1},
            **acc.run("batch_small_closure", storage="f16"))
        del b
        for g in grids:
            lbm.lbm_grid_destroy(g)
    return out


def closure_quality(torch, lbm, wl, N=256, tau0=0.504, T=2048, snap=128, kmax=32, urms=0.03,
                    train_seeds=(11, 12), eval_seeds=(23, 24, 25), train_steps=4000,
                    constants=(0.001, 0.002, 0.004)):
    """The learned closure at the configuration's scale, through the library's
    own dataset and training kernels.  Training: plain fine N^3 periodic
    decaying turbulence at tau0 (k^-5/3 start, u_rms, two seeds), a snapshot
    every `snap` steps up to T, each filtered by r = 2 (the middle level,
    tau_1) and r = 4 (the coarse level, tau_2; one r = 2 sample in eight is
    kept so both levels weigh alike).  Evaluation, three more seeds: the
    3-level slab map (level 0 the central slab) started from the
    box-filtered field runs T / 4 coarsest steps with and without the network
    on levels 1 and 2; the reference is the plain fine run of the same seed,
    box-filtered to each level.  Reported per seed: velocity L2 over the
    voxels of levels 1 and 2 (volume-weighted) without the closure, with the
    network, and with constant corrections d_tau (the best constant is the
    bar a local model should clear); the network's mean gain and its spread
    (sample standard deviation).  tau0 0.504 leaves the coarse levels
    (tau_2 = 0.501) under-damped: over T = 2048 fine steps their error grows
    to ~50 % and a positive d_tau lowers it."""
    t0 = time.time()
    taus = [0.5 + (tau0 - 0.5) / 2 ** l for l in range(3)]
    feats, targs = [], []
    for seed in train_seeds:
        rho, u = wl.turbulence(N, seed=seed, u_rms=urms, kmax=kmax)
        g = lbm.lbm_grid_create_dense((N,) * 3, lbm.physics(tau0, periodic=(1, 1, 1)))
        lbm.lbm_init_equilibrium(g, 0, rho, u)
        del rho, u
        for _ in range(T // snap):
            lbm.lbm_step(g, snap)
            for r, lv, keep in ((2, 1, 8), (4, 2, 1)):
                nc = (N // r) ** 3
                F = torch.empty((nc, 16), dtype=torch.float32, device="cuda")
                Y = torch.empty(nc, dtype=torch.float32, device="cuda")
                lbm.lbm_closure_dataset(g, r, taus[lv], F, Y)
                feats.append(F[::keep].contiguous())
                targs.append(Y[::keep].contiguous())
                del F, Y
        lbm.lbm_grid_destroy(g)
    X = torch.cat(feats).contiguous()
    Y = torch.cat(targs).contiguous()
    del feats, targs
    target_mean = float(Y.mean())
    rng = np.random.default_rng(0)
    th0 = np.concatenate([rng.standard_normal(64 * 16) * np.sqrt(2 / 16), np.zeros(64),
                          rng.standard_normal(64 * 64) * np.sqrt(2 / 64), np.zeros(64),
                          rng.standard_normal(64) * np.sqrt(1 / 64), np.zeros(1)])
    th = torch.from_numpy(th0.astype(np.float32)).cuda()
    t_train = time.time()
    loss = lbm.lbm_closure_train(X, Y, train_steps, 4096, 1e-3, 1, th)
    torch.cuda.synchronize()
    t_train = time.time() - t_train
    n_samples = int(Y.numel())
    del X, Y
    theta = th.cpu().numpy()
    lmap = wl.multires_slab_map(N, 3)
    rows = []
    for seed in eval_seeds:
        rho0, u0 = wl.turbulence(N, seed=seed, u_rms=urms, kmax=kmax)
        g = lbm.lbm_grid_create_dense((N,) * 3, lbm.physics(tau0, periodic=(1, 1, 1)))
        lbm.lbm_init_equilibrium(g, 0, rho0, u0)
        lbm.lbm_step(g, T)
        _, uf = lbm.lbm_get_moments(g, 0)
        lbm.lbm_grid_destroy(g)
        fields = wl.level_fields(rho0, u0, 3)
        judge = [None] + [wl.box_mean(uf, 2 ** lv) for lv in (1, 2)]
        del rho0, u0, uf

        def coarse_error(weights):
            gc = lbm.lbm_grid_create_multires((N,) * 3, 3, lmap, lbm.physics(
                tau0, periodic=(1, 1, 1), closure=int(weights is not None)))
            if weights is not None:
                lbm.lbm_closure_load(gc, weights)
            for lv, (r_, v_) in enumerate(fields):
                lbm.lbm_init_equilibrium(gc, lv, r_, v_)
            lbm.lbm_step(gc, T // 4)
            num = den = 0.0
            for lv in (1, 2):
                _, uc = lbm.lbm_get_moments(gc, lv)
                m = np.isfinite(uc[0])
                ub = judge[lv]
                num += 8.0 ** lv * float(((uc[:, m] - ub[:, m]) ** 2).sum())
                den += 8.0 ** lv * float((ub[:, m] ** 2).sum())
            lbm.lbm_grid_destroy(gc)
            return float(np.sqrt(num / den)) if den > 0 else float("nan")

        plain = coarse_error(None)
        learned = coarse_error(theta)
        const = {}
        for c in constants:
            w = np.zeros(5313, np.float32)
            w[-1] = c
            const[str(c)] = round(coarse_error(w), 5)
        rows.append({"seed": seed, "velocity_l2_plain": round(plain, 5),
                     "velocity_l2_closure": round(learned, 5),
                     "velocity_l2_constant_dtau": const,
                     "gain_pct": round(100 * (1 - learned / plain), 3)})
    gains = np.array([r["gain_pct"] for r in rows])
    best_const = {str(c): round(float(np.mean([100 * (1 - r["velocity_l2_constant_dtau"][str(c)] /
                                                      r["velocity_l2_plain"]) for r in rows])), 3)
                  for c in constants}
    return {"case": f"decaying turbulence, {N}^3 finest box, 3-level slab map, tau_0 {tau0}, "
                    f"u_rms {urms}, kmax {kmax}; levels 1-2 after {T // 4} coarsest steps "
                    f"({T} finest) vs the plain {N}^3 run box-filtered",
            "training_samples": n_samples, "train_steps": train_steps,
            "train_seconds": round(t_train, 2), "final_loss": float(f"{loss:.4e}"),
            "target_mean_dtau": float(f"{target_mean:.4e}"),
            "per_seed": rows, "gain_pct_mean": round(float(gains.mean()), 3),
            "gain_pct_std": round(float(gains.std(ddof=1)), 3) if len(gains) > 1 else None,
            "constant_dtau_gain_pct_mean": best_const,
            "seconds": round(time.time() - t0, 1), "theta": theta}


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    from paper_2503_07898_gb300 import binding as lbm
    from paper_2503_07898_gb300 import build as lbm_build
    from paper_2503_07898_gb300 import workloads as wl
    lbm_build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    n = args.n
    dims = (n, n, n)
    flags, bc = wl.cavity(n)
    tau = 0.515
    stream = torch.cuda.Stream()
    g = lbm.lbm_grid_create_dense(dims, lbm.physics(tau, storage=args.storage,
                                                    schedule=args.schedule), stream=stream)
    lbm.lbm_set_boundary(g, 0, flags, None, np.array([0.05, 0, 0, 1.0], np.float32))
    info = lbm.lbm_get_info(g)
    n_upd = info["n_updated"][0]
    lbm.lbm_init_equilibrium(g, 0, None, None)
    variant, variant_ms = lbm.lbm_autotune(g, 20) if args.variant == "auto" else (
        {"vec16": 0, "scalar": 1, "vec8": 2, "vec4": 3}[args.variant], None)
    lbm.lbm_set_variant(g, variant)
    acc = Accuracy(lbm, wl)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    lbm.lbm_step(g, args.warmup, stream)
    barrier()
    # timed region (A): K steps, events on the launching stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        barrier()
        e0.record(stream)
        lbm.lbm_step(g, args.steps, stream)
        e1.record(stream)
        e1.synchronize()
        barrier()
    ms = max_over_ranks(dist, e0.elapsed_time(e1), "cuda")
    value = job_glups(world, n_upd, args.steps, ms * 1e-3)

    # pass (B): per-kernel CUDA events for the roofline of the dominant kernel
    kb = min(args.steps, 200)
    lbm.lbm_profile(g, 1)
    lbm.lbm_step(g, kb, stream)
    stats = lbm.lbm_profile_read(g)
    lbm.lbm_profile(g, 0)
    launches_per_step = sum(s["launches"] for s in stats.values()) / kb
    top = max(stats, key=lambda k: stats[k]["total_ms"])
    st = stats[top]
    bpu = BYTES_PER_UPDATE[args.storage]
    avg_ms = st["total_ms"] / st["launches"]
    units = st["units"] / st["launches"]
    achieved = bpu * units / (avg_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    tr = NCU_TRAFFIC.get((top, args.storage))
    traffic = tr["bytes_per_launch"] if tr and tr["src_sha"] == src_hash() else None
    shares = {k: round(v["total_ms"] / sum(x["total_ms"] for x in stats.values()), 4)
              for k, v in stats.items()}

    # schedule / storage variants on the same workload (context lines)
    variants = {}
    if not args.no_variants:
        # velocity error of each variant against an FP32 disaggregated run of
        # the same steps (FP32 itself matches the FP64 oracle to 1e-5 in the
        # parity tests): L2 = sqrt(sum |u - u_f32|^2 / sum |u_f32|^2) over the
        # updated voxels, computed on the device
        kv = min(args.steps, 200)
        gr = lbm.lbm_grid_create_dense(dims, lbm.physics(tau), stream=stream)
        lbm.lbm_set_boundary(gr, 0, flags, None, np.array([0.05, 0, 0, 1.0], np.float32))
        lbm.lbm_init_equilibrium(gr, 0, None, None)
        lbm.lbm_step(gr, 20 + kv, stream)
        torch.cuda.synchronize()
        rho_d = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        u_ref = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
        u_var = torch.empty_like(u_ref)
        lbm.lbm_get_moments(gr, 0, rho_d, u_ref)
        lbm.lbm_grid_destroy(gr)
        upd = torch.from_numpy(((flags & 7) == 0) | ((flags & 7) == 2)).cuda()
        u_den = float((u_ref[:, upd] ** 2).sum())
        for name, kw in (("monolithic_f32", dict(storage="f32", schedule="monolithic")),
                         ("disaggregated_f16", dict(storage="f16", schedule="disaggregated")),
                         ("disaggregated_bf16", dict(storage="bf16", schedule="disaggregated")),
                         ("disaggregated_f32_d3q27", dict(storage="f32", schedule="disaggregated",
                                                          lattice=27))):
            q = kw.get("lattice", 19)
            if kw["storage"] == args.storage and kw["schedule"] == args.schedule and q == 19:
                continue
            gv = lbm.lbm_grid_create_dense(dims, lbm.physics(tau, **kw), stream=stream)
            lbm.lbm_set_boundary(gv, 0, flags, None, np.array([0.05, 0, 0, 1.0], np.float32))
            lbm.lbm_init_equilibrium(gv, 0, None, None)
            gv_variant, gv_ms = lbm.lbm_autotune(gv, 20)
            lbm.lbm_step(gv, 20, stream)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            lbm.lbm_step(gv, kv, stream)
            a1.record(stream)
            a1.synchronize()
            vms = a0.elapsed_time(a1)
            lbm.lbm_get_moments(gv, 0, rho_d, u_var)
            l2 = (float(((u_var - u_ref)[:, upd] ** 2).sum()) / u_den) ** 0.5
            vbpu = BYTES_PER_UPDATE[kw["storage"]] * q // 19
            variants[name] = {"GLUPS": round(n_upd * kv / (vms * 1e-3) / 1e9, 3),
                              "roofline_frac": round(n_upd * kv * vbpu / (vms * 1e-3) / 1e9 / peak, 4),
                              "bytes_per_update": vbpu,
                              ("velocity_l2_vs_f32" if q == 19 else "velocity_l2_vs_d3q19_f32"):
                                  float(f"{l2:.3e}"),
                              "l2_vs_f32_after_steps": 20 + kv,
                              "kernel_variant": lbm.VARIANT_NAMES[gv_variant],
                              "autotune_ms_per_step": {lbm.VARIANT_NAMES[k]: round(t, 5)
                                                       for k, t in enumerate(gv_ms) if t > 0}}
            variants[name].update(acc.run(f"cavity48_q{q}", storage=kw["storage"],
                                          schedule=kw["schedule"], variant=gv_variant))
            lbm.lbm_grid_destroy(gv)
        del rho_d, u_ref, u_var

    workloads = {}
    if args.workloads != "none" and rank == 0:
        which = ("sparse", "multires", "batch", "closure") if args.workloads == "all" else tuple(
            args.workloads.split(","))
        theta = None
        quality = None
        if "closure" in which:
            quality = closure_quality(torch, lbm, wl)
            theta = quality.pop("theta")
        workloads = measure_workloads(torch, lbm, wl, stream, peaks()[0], min(args.steps, 100),
                                      which, acc, theta, args.batch_cases)
        if quality is not None:
            workloads["learned_closure_quality"] = quality

    # end to end through the C ABI with pinned host buffers: init from host
    # (rho, u), K steps, moments back to host
    nv = n ** 3
    rho_h = torch.ones(nv, dtype=torch.float64).pin_memory()
    u_h = torch.zeros(3 * nv, dtype=torch.float64).pin_memory()
    rho_o = torch.empty(nv, dtype=torch.float64).pin_memory()
    u_o = torch.empty(3 * nv, dtype=torch.float64).pin_memory()
    barrier()
    t0 = time.perf_counter()
    lbm.lbm_init_equilibrium(g, 0, rho_h, u_h)
    lbm.lbm_step(g, args.steps, stream)
    lbm.lbm_get_moments(g, 0, rho_o, u_o)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0, "cuda")
    e2e = {"value": job_glups(world, n_upd, args.steps, e2e_s), "unit": "GLUPS",
           "h2d_bytes_per_step": 4 * nv * 8, "d2h_bytes_per_step": 4 * nv * 8,
           "lbm_steps_per_step": args.steps,
           "what": "one call sequence: lbm_init_equilibrium(host rho,u) + lbm_step(K) + "
                   "lbm_get_moments(host) from/to pinned memory"}
    assert np.isfinite(rho_o.numpy()).all()

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_line()
        line = {
            "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.storage, "data": "synthetic",
            "config": {"workload": f"cavity{n} dense D3Q19 lid-driven cavity", "dims": list(dims),
                       "tau": tau, "lid_u": 0.05, "collision": "bgk", "storage": args.storage,
                       "schedule": args.schedule, "updated_voxels": n_upd,
                       "variant": lbm.VARIANT_NAMES[variant],
                       "autotune_ms_per_step": (None if variant_ms is None else
                                                {lbm.VARIANT_NAMES[k]: round(t, 5)
                                                 for k, t in enumerate(variant_ms) if t > 0}),
                       "l2": "inputs larger than L2 (population state "
                             f"{2 * info['population_bytes'][0] / 1e9:.2f} GB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak,
                         "peak_kind": f"{peak_kind} (copy, burst)", "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "bytes_per_update": bpu, "units_per_launch": units,
                         "avg_launch_ms": avg_ms, "kernel_time_share": shares},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clk.summary(),
            "accuracy": acc.run("cavity48_q19", storage=args.storage, schedule=args.schedule,
                                variant=variant),
            "accuracy_cases": acc.cases_used(),
            "variants": variants,
            "workloads": workloads,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    lbm.lbm_grid_destroy(g)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--schedule", default="disaggregated", choices=["disaggregated", "monolithic"])
    ap.add_argument("--variant", default="auto", choices=["auto", "vec16", "scalar", "vec8", "vec4"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-cases", type=int, default=128,
                    help="cases of the serving-batch workload (its first n of the 128)")
    ap.add_argument("--workloads", default="all",
                    help="all | none | comma list of sparse,multires,batch,closure "
                         "(turbulence / cavity: one of the two multires workloads)")
    ap.add_argument("--cpu-sample", nargs=3, type=int, metavar=("N", "STEPS", "WARMUP"),
                    help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_sample:
        cpu_sample(*args.cpu_sample)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
