"""Host-side logic of bench.py, on the CPU: the roofline figures it derives from a
device-time profile (fraction of the peak, traffic per launch, choice of the dominant
family) and the reference arm's JSON line, which times the oracle."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
import synth  # noqa: E402

PEAKS = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1500.0, "sm_max_mhz": 2000.0}


def _prof(dhop_ms, tc_ms, ab_ms):
    return {"eloc/links/k_dhop": (12, dhop_ms), "eloc/links/k_tgemm_tc": (6, tc_ms),
            "eloc/abacus/k_ab_layer": (8, ab_ms)}


def test_roofline_fractions_and_traffic():
    desc = synth.CONFIGS["lrtfim_n128"]["desc"]
    N, B, steps = 128, 64, 2
    fam = bench.kernel_rooflines(_prof(40.0, 30.0, 5.0), steps, desc, N, B, PEAKS, "test")
    r = fam["links_dhop"]
    byts = bench.dhop_bytes(N, desc.L, desc.d, B) * steps
    assert r["achieved"] == pytest.approx(byts / 40e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / PEAKS["hbm_gbs"])
    assert r["ms_per_launch"] == pytest.approx(40.0 / 12)
    ratio = bench.DRAM_PER_UNIT["links_dhop"]
    assert r["traffic"] == (None if ratio is None else pytest.approx(ratio * byts / 12))
    t = fam["links_tgemm_tc"]
    flops = bench.link_conv_flops(N, desc.L, desc.d, B) * steps
    assert t["achieved"] == pytest.approx(flops / 30e-3 / 1e12)
    assert t["peak"] == pytest.approx(PEAKS["bf16_tflops_sustained"] / 3)
    a = fam["abacus"]
    P = (desc.L - 1) * (desc.L - 2) // 2
    ab = bench.abacus_unique_bytes(N, desc.L, desc.d, desc.dout, desc.w, P, B) * steps
    assert a["achieved"] == pytest.approx(ab / 5e-3 / 1e9)


@pytest.mark.parametrize("times,kernel", [((40.0, 30.0, 5.0), "k_dhop"), ((10.0, 30.0, 5.0), "k_tgemm_tc"),
                                          ((1.0, 2.0, 5.0), "k_ab_layer")])
def test_roofline_picks_the_family_with_the_most_device_time(times, kernel):
    desc = synth.CONFIGS["lrtfim_n128"]["desc"]
    main, fam = bench.roofline(_prof(*times), 1, desc, 128, 64, PEAKS, "test", None)
    assert main["kernel"] == kernel
    assert main["bound"] in ("hbm", "tensor")


def test_algorithmic_units_scale_with_the_batch():
    d = synth.CONFIGS["lrtfim_n128"]["desc"]
    for f in (lambda B: bench.dhop_bytes(128, d.L, d.d, B), lambda B: bench.link_conv_flops(128, d.L, d.d, B),
              lambda B: bench.bandconv_bytes(128, d.L, d.d, d.w, B),
              lambda B: bench.bandconv_gen_flops(128, d.L, d.d, d.w, B)):
        assert f(6) == 3 * f(2) > 0


def test_reference_arm_json_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3",
                          "--ref-samples", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "flip ratios/s" and line["value"] > 0
    assert line["steps"] == 1 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
