"""Host-side legs of the benchmark that need no GPU: the oracle's CPU
baseline sample runs on every workload the benchmark accepts (each sampled
subdomain has enough local realizations, the batched workload samples its
batch), and the workload descriptions carry their sizes."""

import pytest

import sfb_workloads as W


@pytest.mark.parametrize("workload", ["tiny", "medium", "batched"])
def test_cpu_baseline_sample_runs_on_every_workload(workload):
    import bench
    cb = bench.cpu_baseline_sample(n_items=16, n_pts=4, workload=workload)
    assert cb["value"] > 0 and cb["cores"] == 1 and cb["kind"] == "oracle"
    n_batch = W.ALL[workload]().get("n_batch")
    if n_batch:
        assert ("of %d points" % n_batch) in cb["sample"]


def test_reference_arm_names_the_workload():
    import argparse
    import bench
    out = bench.run_reference(argparse.Namespace(warmup=0, steps=1, workload="tiny"))
    assert out["impl"] == "reference" and out["config"]["workload"].startswith("tiny")
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["value"] == out["cpu_baseline"]["value"]


def test_cpu_baseline_all_cores_runs_spawned_workers():
    """The all-cores oracle baseline (one spawned process per core) returns a
    throughput with the core count it used, not an error record."""
    import bench
    cb = bench.cpu_baseline_all_cores(workload="tiny", items_per_core=1, pts_per_core=4, cores=2)
    assert "error" not in cb, cb
    assert cb["value"] > 0 and cb["cores"] == 2 and cb["kind"] == "oracle"


def test_host_cores_is_bounded():
    import bench
    n = bench.host_cores()
    assert 1 <= n <= 32
    assert bench.host_cores(cap=1) == 1
