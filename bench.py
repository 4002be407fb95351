"""Benchmark: D3Q19 GLUPS and fraction of the HBM roofline on one GB300.

Default workload (the lid-driven cavity the metric is quoted on): dense
256^3 D3Q19, FP32 storage, BGK tau = 0.515, regularized lid u = 0.05 on the
top plane, bounce-back on the other walls, disaggregated schedule (lean
interior kernel + regularized lid kernel).  One bench step = one lattice
time step over the whole grid.  The 2.55 GB population state is ~20x the
L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  --impl reference times the FP64 oracle (the plain
numpy program the CUDA path is checked against) on the host cores.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_UPDATE = {"f32": 152, "f16": 76, "bf16": 76}   # 19 loads + 19 stores
METRIC = "D3Q19 GLUPS & % HBM roofline, FP32 vs FP16-store/learned at stated error"

# DRAM traffic of the dominant kernel from an ncu capture (profiles/), valid
# only while the kernel sources hash to the recorded value: the 160^3
# capture of dense_interior (dram__bytes_read.sum + dram__bytes_write.sum,
# 4,070,400 updates per launch) scaled by units to one 256^3 launch
# (16,711,680 updates), profiles/dense_interior_cavity160_ncu.md; keyed by
# kernel and storage (the FP16 capture: dense_interior_f16_cavity160_ncu.md).
NCU_TRAFFIC = {("dense_interior", "f32"): {"bytes_per_launch": 2.351797e+09, "src_sha": "d62c038efe78398d"},
               ("dense_interior", "f16"): {"bytes_per_launch": 1.118711e+09, "src_sha": "d62c038efe78398d"}}


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

def oracle_cavity_glups(n, steps, tau=0.515, u_lid=0.05):
    """The FP64 oracle as it stands on an n^3 cavity (same physics as the
    GPU workload); returns (GLUPS, seconds)."""
    from oracle import lbm as olbm
    from paper_2503_07898_gb300 import workloads as wl
    flags, bc = wl.cavity(n, u_lid=u_lid)
    f = olbm.init_equilibrium(np.ones((n, n, n)), np.zeros((3, n, n, n)))
    f = olbm.step(f, flags, tau, bc=bc)          # warm-up
    c0 = time.process_time()
    t0 = time.perf_counter()
    for _ in range(steps):
        f = olbm.step(f, flags, tau, bc=bc)
    dt = time.perf_counter() - t0
    cores = (time.process_time() - c0) / dt      # threads numpy/BLAS actually kept busy
    return n ** 3 * steps / dt / 1e9, dt, round(cores, 1)


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
    from oracle import lbm as olbm  # noqa: F401
    oracle_cavity_glups(n, max(1, args.warmup))
    value, dt, cores = oracle_cavity_glups(n, args.steps)
    sample = f"{n}^3 cavity window of the 256^3 workload, tau 0.515, lid 0.05, numpy FP64"
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


def measure_workloads(torch, lbm, wl, stream, peak, steps, which, n_batch=128):
    """GLUPS of the other layouts of the method on their full-size inputs
    (context lines of the same metric; each timed after 3 warm-up steps)."""
    STAGED = lbm.LBM_VARIANT_STAGED
    out = {}
    # a closure network of the trained one's size and scale (random weights:
    # the cost of inference does not depend on their values)
    rng = np.random.default_rng(0)
    theta = np.concatenate([rng.standard_normal(1024) * 0.35, np.zeros(64),
                            rng.standard_normal(4096) * 0.18, np.zeros(64),
                            rng.standard_normal(64) * 1e-3, np.zeros(1)]).astype(np.float32)
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
            out[key] = res
    if "multires" in which or "turbulence" in which:
        lmap = wl.multires_slab_map()
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
                lbm.lbm_init_equilibrium(g, l, None, None)
            lbm.lbm_step(g, 3, stream)
            ms = _time_steps(torch, lbm, lambda n: lbm.lbm_step(g, n, stream), stream,
                             max(1, steps // 4))
            glups = ups * max(1, steps // 4) / (ms * 1e-3) / 1e9
            bpu = (76 if kw.get("storage") == "f16" else 152) * kw.get("lattice", 19) // 19
            res[name] = {"GLUPS": round(glups, 3), "roofline_frac": round(glups * bpu / peak, 4)}
            lbm.lbm_grid_destroy(g)
        res["updates_per_coarsest_step"] = ups
        out["turbulence_256_3level"] = res
    cavities = ((384, 3, (2, 2), (("fused_f32", dict()), ("fused_f32_staged", dict(variant=STAGED)),
                                  ("unfused_f32", dict(schedule="monolithic")),
                                  ("fused_f16", dict(storage="f16")))),
                (512, 4, (1, 1, 1), (("fused_f32", dict()),
                                     ("unfused_f32", dict(schedule="monolithic")))))
    for n, nlev, shells, cases in (cavities if ("multires" in which or "cavity" in which) else ()):
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
        out[f"serving_batch_{n_batch}_f16"] = {"GLUPS": round(glups, 3),
                                        "roofline_frac": round(glups * 76 / peak, 4),
                                        "updated_voxels": info["n_updated"],
                                        "ctas_per_sm": k, "launches_per_step": 1}
        # the learned closure on the cases whose largest edge is <= 64
        lbm.lbm_batch_closure_load(b, theta, 64)
        n_cl = sum(1 for c in cases if max(c["dims"]) <= 64)
        k, _ = lbm.lbm_batch_autotune(b, 4)
        lbm.lbm_batch_step(b, steps, stream)
        torch.cuda.synchronize()
        ms = _time_steps(torch, lbm, lambda n: lbm.lbm_batch_step(b, n, stream), stream, steps)
        glups = info["n_updated"] * steps / (ms * 1e-3) / 1e9
        out[f"serving_batch_{n_batch}_f16_learned_closure"] = {
            "GLUPS": round(glups, 3), "roofline_frac": round(glups * 76 / peak, 4),
            "closure_cases": n_cl, "max_edge": 64, "ctas_per_sm": k, "launches_per_step": 1}
        del b
        for g in grids:
            lbm.lbm_grid_destroy(g)
    return out


def closure_quality(torch, lbm, wl, N=64, r=4, tau_f=0.504, T=192, kmax=16, urms=0.03):
    """Error of the learned closure, through the library's own dataset and
    training kernels: fine N^3 decaying turbulence at tau_f (two seeds,
    snapshots every 16 steps) gives the training set of a level r times
    coarser; the trained network then runs on that coarse level of a 3-level
    grid (tau_2 = 1/2 + (tau_f - 1/2) / r) started from the box-filtered fine
    field of a third seed.  Reported: velocity L2 against the box-filtered
    fine run after T fine steps, with and without the closure."""
    def box(a):
        *lead, nz, ny, nx = a.shape
        return a.reshape(*lead, nz // r, r, ny // r, r, nx // r, r).mean(axis=(-5, -3, -1))

    tau_c = 0.5 + (tau_f - 0.5) / r
    nc = (N // r) ** 3
    feats, targs = [], []
    t0 = time.time()
    for seed in (11, 12):
        rho, u = wl.turbulence(N, seed=seed, u_rms=urms, kmax=kmax)
        g = lbm.lbm_grid_create_dense((N,) * 3, lbm.physics(tau_f, periodic=(1, 1, 1)))
        lbm.lbm_init_equilibrium(g, 0, rho, u)
        for _ in range(T // 16):
            lbm.lbm_step(g, 16)
            F = torch.empty((nc, 16), dtype=torch.float32, device="cuda")
            Y = torch.empty(nc, dtype=torch.float32, device="cuda")
            lbm.lbm_closure_dataset(g, r, tau_c, F, Y)
            feats.append(F)
            targs.append(Y)
        lbm.lbm_grid_destroy(g)
    X = torch.cat(feats).contiguous()
    Y = torch.cat(targs).contiguous()
    rng = np.random.default_rng(0)
    th0 = np.concatenate([rng.standard_normal(64 * 16) * np.sqrt(2 / 16), np.zeros(64),
                          rng.standard_normal(64 * 64) * np.sqrt(2 / 64), np.zeros(64),
                          rng.standard_normal(64) * np.sqrt(1 / 64), np.zeros(1)])
    th = torch.from_numpy(th0.astype(np.float32)).cuda()
    loss = lbm.lbm_closure_train(X, Y, 4000, 4096, 1e-3, 1, th)
    theta = th.cpu().numpy()
    rho0, u0 = wl.turbulence(N, seed=23, u_rms=urms, kmax=kmax)
    g = lbm.lbm_grid_create_dense((N,) * 3, lbm.physics(tau_f, periodic=(1, 1, 1)))
    lbm.lbm_init_equilibrium(g, 0, rho0, u0)
    lbm.lbm_step(g, T)
    _, uf = lbm.lbm_get_moments(g, 0)
    lbm.lbm_grid_destroy(g)
    ub = box(uf)
    lmap = np.full((N // 32,) * 3, 2, np.uint8)
    errs = {}
    for closure in (0, 1):
        gc = lbm.lbm_grid_create_multires((N,) * 3, 3, lmap,
                                          lbm.physics(tau_f, periodic=(1, 1, 1), closure=closure))
        if closure:
            lbm.lbm_closure_load(gc, theta)
        lbm.lbm_init_equilibrium(gc, 2, box(rho0), box(u0))
        lbm.lbm_step(gc, T // r)
        _, uc = lbm.lbm_get_moments(gc, 2)
        lbm.lbm_grid_destroy(gc)
        errs[closure] = float(np.sqrt(((uc - ub) ** 2).sum() / (ub ** 2).sum()))
    return {"case": f"decaying turbulence, fine {N}^3 tau {tau_f} u_rms {urms} vs the level "
                    f"{r}x coarser (tau {tau_c}) after {T} fine steps",
            "training_samples": int(Y.numel()), "final_loss": float(f"{loss:.4e}"),
            "velocity_l2_plain": round(errs[0], 5), "velocity_l2_closure": round(errs[1], 5),
            "gain_pct": round(100 * (1 - errs[1] / errs[0]), 2),
            "seconds": round(time.time() - t0, 1)}


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
            lbm.lbm_autotune(gv, 20)
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
                              "after_steps": 20 + kv}
            lbm.lbm_grid_destroy(gv)
        del rho_d, u_ref, u_var

    workloads = {}
    if args.workloads != "none" and rank == 0:
        which = ("sparse", "multires", "batch", "closure") if args.workloads == "all" else tuple(
            args.workloads.split(","))
        workloads = measure_workloads(torch, lbm, wl, stream, peaks()[0], min(args.steps, 100),
                                      which, args.batch_cases)
        if "closure" in which:
            workloads["learned_closure_quality"] = closure_quality(torch, lbm, wl)

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
            cn, csteps = 64, 200  # about 10 s of the oracle on the host cores
            cv, cdt, ccores = oracle_cavity_glups(cn, csteps)
            cpu = {"value": cv, "unit": "GLUPS", "cores": ccores, "kind": "oracle",
                   "sample": f"{cn}^3 cavity (tau 0.515, lid 0.05), {csteps} steps, numpy FP64, "
                             f"{cdt:.1f} s"}
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
                         "bytes_per_update": bpu, "units_per_launch": units,
                         "avg_launch_ms": avg_ms, "kernel_time_share": shares},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clk.summary(),
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
    args = ap.parse_args()
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
