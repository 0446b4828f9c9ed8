"""The parts of bench.py's JSON contract that run without a GPU: the reference arm's line
(the oracle on the host cores), the cpu_baseline object and the workload description."""
import io
import json
import types
from contextlib import redirect_stdout

import pytest

import bench
from paper_2505_00097_gb300 import workloads as W


def _tiny():
    s = W.config_headon()
    s.update(N=(16, 2, 32), name="headon_sinhcyl_16x2x32")
    return s


def test_reference_arm_prints_one_contract_line():
    args = types.SimpleNamespace(steps=2, warmup=1, gpus=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, _tiny())
    lines = [x for x in buf.getvalue().splitlines() if x.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["vs_baseline"] is None and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "headon_sinhcyl_16x2x32"
    # the same work as a step of the GPU arm (full integrator steps of the whole grid), described by the
    # same config the GPU arm prints at one replica
    assert "2 full RK4 steps" in cb["sample"]
    assert line["config"]["parallelism"] == "replicas x1" and line["config"]["dt"] > 0


def test_cpu_baseline_object():
    cb = bench.cpu_baseline(_tiny(), 0.3)
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT and cb["value"] > 0 and cb["cores"] >= 1
    assert "RK4 steps" in cb["sample"]
    assert set(cb["diagnostics"]) == {"hamiltonian_ms", "momentum_ms", "psi4_ms", "psi4_modes_ms"}


@pytest.mark.parametrize("name", ["headon", "headon8", "large3d", "single_puncture"])
def test_workload_descriptions(name):
    spec = bench.workload(name)
    c = bench.config_of(spec)
    assert c["workload"] == spec["name"] and c["grid_interior"] == list(spec["N"])
    assert c["fd_order"] == (8 if name == "headon8" else 4)
    assert c["integrator"] == ("SSPRK3" if name == "headon8" else "RK4")
    assert "l2_policy" in c
    if name in bench.F_ALG:
        # a BSSN RHS evaluation with 4th- or 8th-order stencils: a few thousand FLOP per point
        assert 1000 < bench.F_ALG[name] < 10000
