"""bench.py on the CPU: the reference arm's JSON line (the oracle timed on whole coarse
steps of the default workload), the silence of ranks other than 0, and the
cell-update accounting of the workloads (Sigma_l n_l^3 2^l per coarse step)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1812_03191_gb300 import inputs as I  # noqa: E402


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args,
                         capture_output=True, text=True, timeout=600, env=e, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    return [json.loads(l) for l in out.stdout.splitlines() if l.startswith("{")]


def test_default_workload_is_the_precision_configuration():
    """the default bench line is the largest single-GPU configuration: 5 x 128^3"""
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'ap.add_argument("--workload", default="precision"' in src
    assert bench.workload("precision")["name"] == "precision_5x128^3"


def test_reference_arm_line():
    (line,) = _run(["--impl", "reference", "--workload", "nested", "--steps", "1",
                    "--warmup", "3"])
    assert line["impl"] == "reference"
    assert line["metric"] == "cell-updates/s" and line["unit"] == "cell-updates/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["config"]["workload"] == "nested_3x64^3_fp64"
    assert line["ms_per_step"] == pytest.approx(
        1e3 * bench.cell_updates_per_step(I.nested()) / line["value"], rel=1e-9)
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["value"] == line["value"]
    assert cpu["unit"] == line["unit"] and cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    assert _run(["--impl", "reference", "--workload", "nested", "--steps", "1", "--warmup",
                 "3"], env={"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_cell_updates_per_coarse_step():
    """n^3 (1 + 2 + ... + 2^(L-1)): 3 x 64^3 -> 1.835e6, 5 x 128^3 -> 6.50e7"""
    assert bench.cell_updates_per_step(I.nested()) == 64**3 * 7
    assert bench.cell_updates_per_step(I.precision()) == 128**3 * 31
    assert bench.cell_updates_per_step({"n": (8, 8, 16), "n_levels": 2}) == 8 * 8 * 16 * 3


def test_level_step_boxes():
    """one box per level step: level 0 once with margin 4 (5 above); level l >= 1 2^(l-1) times
    per sub-cycle pair, margins 8 then 4, capped at the padded array"""
    cfg = I.nested()
    n, G = cfg["n"], cfg["G"]
    boxes = bench.level_step_boxes(cfg)
    assert len(boxes) == 2 ** cfg["n_levels"] - 1
    assert boxes[0] == (n + 9) ** 3  # level 0: one more element on the upper side
    assert sorted(set(boxes)) == sorted({(n + 9) ** 3, (n + 8) ** 3,
                                         min(n + 16, n + 2 * G) ** 3})


def test_kernel_hbm_table():
    """bytes per launch over the mean box / mean launch time; kinds without a byte
    count are left out"""
    cfg = I.precision()
    boxes = bench.level_step_boxes(cfg)
    mean_box = sum(boxes) / len(boxes)
    kinds = {"source": (10.0, 310), "sweep": (68.5, 930), "dt": (1.5, 100)}
    t = bench.kernel_hbm_table(cfg, kinds, 4, True, 6800.0)
    assert set(t) == {"source", "sweep"}
    gbs = 12 * 4 * mean_box / (10.0 / 310 / 1e3) / 1e9
    assert t["source"]["gbs"] == pytest.approx(gbs, abs=0.1)
    assert t["source"]["frac"] == pytest.approx(gbs / 6800.0, abs=1e-3)
    assert t["sweep"]["gbs"] == pytest.approx(11 * 4 * mean_box / (68.5 / 930 / 1e3) / 1e9,
                                              abs=0.1)


def test_roofline_block_arithmetic():
    """the dominant level-step kernel's roofline: 80 B (FP64) per cell-update of one
    level step of one n^3 level over its mean launch time; traffic = the captured DRAM
    bytes per box element times the mean box; the whole step on the same bytes"""
    cfg = I.precision()
    n = cfg["n"]
    cu = bench.cell_updates_per_step(cfg)
    kinds = {"tmom": (108.0, 1860), "tupdate": (98.0, 1860), "dt": (4.0, 100)}
    m = {"kinds": kinds, "ms": 210.0, "steps": 10}
    r = bench.roofline_block(cfg, m, cu, 8, 6786.2, "measured")
    assert r["kernel"] == "tmom"  # the largest share among the level-step kernels
    avg_s = 108.0 / 1860 / 1e3
    assert r["achieved"] == pytest.approx(80 * n**3 / avg_s / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6786.2)
    boxes = bench.level_step_boxes(cfg)
    per_elem = bench.TRAFFIC_PER_ELEM[(cfg["name"], 8, "tmom")]
    assert r["traffic"] == pytest.approx(per_elem * sum(boxes) / len(boxes))
    # the capture's 34.9 B per box element of the 80^3 launches
    assert per_elem == pytest.approx(34.9, abs=0.05)
    assert r["step"]["frac"] == pytest.approx(cu * 80 / (21.0 / 1e3) / 1e9 / 6786.2)
    assert r["share_of_kernel_time"] == pytest.approx(108.0 / 210.0)
    # an FP32 run has no traffic figure for tmom and takes 40 B
    r32 = bench.roofline_block(cfg, m, cu, 4, 6786.2, "measured")
    assert r32["traffic"] is None
    assert r32["achieved"] == pytest.approx(r["achieved"] / 2)
