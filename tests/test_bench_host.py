"""Host logic of bench.py: the synthesis count behind syntheses/s and the
roofline, the flop model's structure, and the reference arm's JSON line
(the FP64 oracle on the host cores; no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _walk_schedule(npop, ngen, nsamp):
    """Fitness evaluations of one pixel, generation by generation: the
    initial population, every child of generations 1..ngen, and the worst
    half again after generation t whenever t is a multiple of nsamp and
    t < ngen (Section 5.6 restarts)."""
    n = npop
    for t in range(1, ngen + 1):
        n += npop
        if nsamp > 0 and t % nsamp == 0 and t < ngen:
            n += npop // 2
    return n


@pytest.mark.parametrize("npop,ngen,nsamp", [(128, 200, None), (64, 100, None), (128, 300, None),
                                             (32, 16, None), (64, 3, None), (64, 12, 5), (256, 7, 0)])
def test_syntheses_per_pixel_matches_the_schedule(npop, ngen, nsamp):
    ns = ngen // 4 if nsamp is None else nsamp
    assert bench.syntheses_per_pixel(npop, ngen, nsamp) == _walk_schedule(npop, ngen, ns)


def test_syntheses_per_pixel_of_the_benchmark():
    # 128 x 201 evaluations plus three restarts (t = 50, 100, 150) of 64
    assert bench.syntheses_per_pixel(128, 200) == 25920


def test_flop_model_structure():
    for nl in (1, 2, 4):
        fm = bench.flop_model(nl)
        # the cheaper a w(z) branch, the fewer flops it is credited with
        assert fm["weideman"] > fm["mid"] > fm["cf"] > fm["even2"] > fm["far"] > 0
        assert fm["point"] == pytest.approx(16.0 * nl + 71.0)


def test_reference_arm_json_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "pixels/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["n_gpus"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "pixels/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
