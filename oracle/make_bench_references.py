"""Write the FP64 oracle's velocities for the benchmark's accuracy cases.

Test infrastructure, run by hand (python -m oracle.make_bench_references);
it calls only this package and the seeded input generators.  For every
reduced case of `workloads.accuracy_cases()` (a small case of the same shape
as a benchmark workload) the oracle runs the case whole in FP64 and the
velocity u = sum f c / sum f at the case's sampled updated voxels is stored,
with the sample indices, in tests/golden/bench_velocity_references.npz.  The
benchmark runs the same cases through the library with each line's storage,
schedule and kernel variant and reports the relative velocity L2 error over
those voxels; it never executes the oracle itself.

Readings: boundary values reach the oracle rounded to FP32, as the library
stores them; a closure network reaches it with W1, W2 and W3 rounded to BF16
(nearest even), the form the collision kernels hold (biases stay FP32).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import closure as ocl  # noqa: E402
from oracle import lbm as olbm  # noqa: E402
from oracle import multires as omr  # noqa: E402
from paper_2503_07898_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "bench_velocity_references.npz")


def fp32_bc(flags, bc):
    if bc is None:
        return None
    out = np.array(bc, dtype=np.float64, copy=True)
    t = flags & 7
    sel = (t == wl.VELOCITY) | (t == wl.PRESSURE)
    out[:, sel] = bc[:, sel].astype(np.float32).astype(np.float64)
    return out


def bf16_weights(theta):
    """W1, W2, W3 rounded to BF16 (nearest even), biases unchanged."""
    th = np.asarray(theta, np.float32)
    bits = th.view(np.uint32).astype(np.uint64)
    rounded = (((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16).astype(np.uint32)
    bf = rounded.view(np.float32).astype(np.float64)
    out = th.astype(np.float64)
    for sl in (slice(0, 1024), slice(1088, 5184), slice(5248, 5312)):
        out[sl] = bf[sl]
    return out


def velocity_at(f, idx):
    _, u = olbm.state_moments(f)
    return u.reshape(3, -1)[:, idx]


def run_case(case):
    """List of (3, n_samples) velocities, one per sample set of the case."""
    samples = wl.accuracy_samples(case)
    per = tuple(bool(p) for p in case["periodic"])
    if case["kind"] in ("dense", "sparse"):
        rho, u = case["fields"][0]
        f = olbm.init_equilibrium(rho, u, case["flags"], q=case["q"])
        obc = fp32_bc(case["flags"], case["bc"])
        for _ in range(case["steps"]):
            f = olbm.step(f, case["flags"], case["tau"], periodic=per, bc=obc)
        return [velocity_at(f, samples[0])]
    if case["kind"] == "batch":
        out = []
        th = None if case.get("theta") is None else bf16_weights(case["theta"])
        for c, idx in zip(case["cases"], samples):
            rho, u = wl.batch_case_fields(c)
            f = olbm.init_equilibrium(rho, u, c["flags"])
            if th is None:
                f = olbm.run(f, c["flags"], c["tau"], case["steps"], periodic=per)
            else:
                f = ocl.run(f, c["flags"], c["tau"], th, case["steps"], periodic=per)
            out.append(velocity_at(f, idx))
        return out
    nx = case["dims"][0]
    cell = nx // case["level_map"].shape[2]
    th = None if case.get("theta") is None else bf16_weights(case["theta"])
    o = omr.MultiRes(case["level_map"], case["n_levels"], cell, case["tau"], theta=th,
                     periodic=per, flags0=case["flags"],
                     bc0=fp32_bc(case["flags"], case["bc"]), q=case["q"])
    for lv, (rho, u) in enumerate(case["fields"]):
        o.init_equilibrium(lv, rho, u)
    o.run(case["steps"])
    return [velocity_at(o.f[lv], samples[lv]) for lv in range(case["n_levels"])]


def main(names=None):
    cases = wl.accuracy_cases()
    old = dict(np.load(OUT)) if os.path.exists(OUT) else {}
    manifest = json.loads(str(old.pop("manifest"))) if "manifest" in old else {}
    data = dict(old)
    for name, case in cases.items():
        if names and name not in names:
            continue
        t0 = time.time()
        us = run_case(case)
        for k, (u, idx) in enumerate(zip(us, wl.accuracy_samples(case))):
            data[f"{name}/u{k}"] = u.astype(np.float32)
            data[f"{name}/idx{k}"] = idx.astype(np.int32)
        manifest[name] = {"what": case["what"], "steps": case["steps"], "sets": len(us)}
        print(f"{name}: {time.time() - t0:.1f} s", flush=True)
    data["manifest"] = np.array(json.dumps(manifest, sort_keys=True))
    np.savez_compressed(OUT, **data)


if __name__ == "__main__":
    main(sys.argv[1:] or None)
