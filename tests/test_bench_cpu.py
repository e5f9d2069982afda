"""bench.py's reference arm (the FP64 oracle timed on the host cores) runs
without a GPU and prints the benchmark contract's JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--chi", "6", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in KEYS:
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "sweep/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "sweep/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert "chi=6" in line["config"]["workload"]


def test_reported_planner_widths_match_the_planner():
    """bench.py reports which GEMM shapes the autotuner moved by comparing
    each planned width with its copy of the planner's rule; the copy must
    agree with every untuned plan."""
    sys.path.insert(0, ROOT)
    import bench
    import paper_1906_12030_gb300 as m

    m.mera_autotune_reset()
    for name in ("tf32", "bf16", "bf16x3", "bf16x6"):
        prec = m.PRECS[name]
        for chi_b, chi_t in ((4, 16), (16, 16), (8, 8), (3, 5)):
            for op in (m.OP_ASCEND, m.OP_DESCEND, m.OP_ENV_U, m.OP_ENV_W):
                for dg in m.mera_plan_json(op, chi_b, chi_t, prec)["diagrams"]:
                    for st in dg["steps"]:
                        if st["kind"] == "gemm":
                            assert st["bn"] == bench._heuristic_bn(name, st["N"]), (name, op, st["N"])
