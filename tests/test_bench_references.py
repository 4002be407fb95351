"""The stored oracle velocities the benchmark compares against are current:
one entry per sample set of every accuracy case, at the sampled voxels the
seeded inputs give today, finite and nonzero (a change to a case's inputs
without re-running oracle/make_bench_references.py fails here)."""
import json
import os

import numpy as np
import pytest

from paper_2503_07898_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REFS = os.path.join(ROOT, "tests", "golden", "bench_velocity_references.npz")


@pytest.fixture(scope="module")
def refs():
    return dict(np.load(REFS))


def test_every_case_has_current_references(refs):
    manifest = json.loads(str(refs["manifest"]))
    cases = wl.accuracy_cases()
    assert set(manifest) == set(cases)
    for name, case in cases.items():
        samples = wl.accuracy_samples(case)
        assert manifest[name]["sets"] == len(samples)
        assert manifest[name]["steps"] == case["steps"]
        for k, idx in enumerate(samples):
            assert np.array_equal(refs[f"{name}/idx{k}"], idx), (name, k)
            u = refs[f"{name}/u{k}"]
            assert u.shape == (3, len(idx))
            assert np.all(np.isfinite(u)) and np.abs(u).max() > 0, (name, k)
