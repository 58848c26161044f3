"""bench.py's reference arm on CPU: the oracle timed on the host cores prints one JSON
line with the contract's keys, for the same metric and workload as the GPU arm; under
torchrun only rank 0 prints."""
import contextlib
import io
import json
import os

import bench


def _run(argv, env=None):
    old = {k: os.environ.get(k) for k in (env or {})}
    os.environ.update(env or {})
    try:
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            rc = bench.main(argv)
        return rc, buf.getvalue()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def test_reference_arm_prints_the_contract_line():
    import time
    t0 = time.perf_counter()
    rc, out = _run(["--impl", "reference", "--steps", "3", "--warmup", "3", "--workload", "small",
                    "--reference-draws-per-core", "2"])
    wall = time.perf_counter() - t0
    assert rc == 0
    line = json.loads(out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "whitened injections/sec" and line["unit"] == "injections/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 3 and line["warmup"] == 3 and line["dtype"] == "f64"
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"]
    assert "spawned processes" in cpu["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["global_batch"] == 64 and line["config"]["seq_len"] == 2048
    # every draw the line reports was timed: the steps' time fits in the run's own wall time
    assert line["steps"] * line["ms_per_step"] * 1e-3 <= wall
    # the same config object as the GPU arm prints
    import argparse
    import workloads
    assert line["config"] == bench.bench_config(workloads.workload("small"), argparse.Namespace(background_every=16), 1)


def test_reference_arm_is_silent_on_other_ranks():
    rc, out = _run(["--impl", "reference", "--steps", "3", "--warmup", "3"], env={"RANK": "1"})
    assert rc == 0 and out.strip() == ""


def test_warmup_below_three_is_refused():
    import pytest
    with pytest.raises(SystemExit):
        bench.main(["--impl", "reference", "--steps", "3", "--warmup", "2"])
