"""bench.py's reference arm (the FP64 oracle timed on the host cores) runs
without a GPU and without the CUDA library, and prints the benchmark
contract's JSON line with the same config as the native arm."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")

# runs the reference arm in a fresh interpreter and reports whether any part
# of the CUDA library's package was imported
_DRIVER = """
import sys
sys.argv = ["bench.py"] + sys.argv[1:]
import bench
bench.main()
print("LOADED=" + str(any(k.startswith("paper_1906_12030_gb300") for k in sys.modules)))
"""


def _reference(chi, steps=2, warmup=1):
    out = subprocess.run([sys.executable, "-c", _DRIVER, "--impl", "reference", "--chi", str(chi), "--steps",
                          str(steps), "--warmup", str(warmup)], cwd=ROOT, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert "LOADED=False" in out.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("chi,whole", [(8, True), (12, False)])
def test_reference_arm_prints_the_contract_line(chi, whole):
    line = _reference(chi)
    for k in KEYS:
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "sweep/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "sweep/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["extrapolated"] is (not whole)
    # the same workload description as the native arm
    assert line["config"] == bench._config(chi)
    assert f"chi={chi}" in line["config"]["workload"]
    if whole:  # a whole sweep per step: value and ms_per_step agree
        assert abs(line["value"] * line["ms_per_step"] / 1e3 - 1.0) < 1e-9


def test_diagram_flop_table_matches_the_planner():
    """bench.py's copy of the per-diagram flops (so that the reference arm
    needs no library) agrees with the library's planner for every entry."""
    import paper_1906_12030_gb300 as m

    ops = {"ascend": m.OP_ASCEND, "descend": m.OP_DESCEND, "env_u": m.OP_ENV_U, "env_w": m.OP_ENV_W}
    for (cb, ct), per in bench.DIAGRAM_FLOPS.items():
        for name, op in ops.items():
            assert m.mera_flops(op, cb, ct) == bench.N_DIAGRAMS[name] * per, (cb, ct, name)
    assert bench._sweep_flops(16) == pytest.approx(1.98e13, rel=0.01)
    assert bench._sweep_flops(32) == pytest.approx(7.49e15, rel=0.01)


def test_reported_planner_widths_match_the_planner():
    """bench.py reports which GEMM shapes the autotuner moved by comparing
    each planned width with its copy of the planner's rule; the copy must
    agree with every untuned plan."""
    import paper_1906_12030_gb300 as m

    m.mera_autotune_reset()
    for name in ("tf32", "bf16", "bf16x3", "bf16x6", "oz3", "oz4"):
        prec = m.PRECS[name]
        for chi_b, chi_t in ((4, 16), (16, 16), (8, 8), (3, 5), (12, 12), (24, 24)):
            for op in (m.OP_ASCEND, m.OP_DESCEND, m.OP_ENV_U, m.OP_ENV_W):
                for dg in m.mera_plan_json(op, chi_b, chi_t, prec)["diagrams"]:
                    for st in dg["steps"]:
                        if st["kind"] == "gemm":
                            assert st["bn"] == bench._heuristic_bn(name, st["N"]), (name, op, st["N"])
