"""The benchmark's reference arm (the oracle on the host cores) prints one
JSON line with the keys of the benchmark contract (no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--shape", "300", "240", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e", "impl"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["m"] == 300 and d["config"]["n"] == 240
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_stage_roofline_arithmetic():
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1600.0,
             "fp64_tflops": 1.0}
    m = n = 8192
    l, q, d = 110, 1, 2
    work = bench._class_work(m, n, l, q, d, "bf16x3")
    # one step, each class taking 1 ms
    prof = {k: (1.0, 1) for k in work}
    sr = bench._stage_roofline("bf16x3", m, n, l, q, d, prof, 1, peaks)
    pa = sr["products_with_A"]
    # 4 passes over the BF16 pair (4 bytes per element) in 1 ms
    assert pa["bound"] == "hbm"
    assert abs(pa["achieved_gbs"] - 4 * 4.0 * m * n / 1e-3 / 1e9) < 1e-6
    assert abs(pa["frac"] - pa["achieved_gbs"] / 6000.0) < 1e-12
    # three tensor-core products per pass, 2 m n l flops each
    assert abs(pa["tensor_tflops"] - 3 * 4 * 2.0 * m * n * l / 1e-3 / 1e12) < 1e-6
    assert abs(pa["tensor_frac"] - pa["tensor_tflops"] / 1600.0) < 1e-12
    cp = sr["cpqr_of_B"]
    assert cp["bound"] == "alu"
    assert abs(cp["achieved_tflops"] - 2.0 * n * l * (l + 1) / 1e-3 / 1e12) < 1e-9
    assert abs(cp["frac"] - cp["achieved_tflops"] / 1.0) < 1e-12  # the measured FP64 rate
    # the assembly at d <= 2 is the product Q = V Q_B only (P is a row scatter);
    # in the mixed forms it runs as digit products: an FP64-equivalent rate
    a2 = sr["assembly"]
    assert a2["bound"].startswith("tensor")
    assert abs(a2["fp64_equiv_tflops"] - 2.0 * m * l * l / 1e-3 / 1e12) < 1e-9
    assert abs(a2["x_fp64_units"] - a2["fp64_equiv_tflops"]) < 1e-12
    sr3 = bench._stage_roofline("fp64", m, n, l, q, 3, prof, 1, peaks)
    assert abs(sr3["assembly"]["achieved_tflops"] - 2.0 * (m + n) * l * l / 1e-3 / 1e12) < 1e-9
    # FP64TC: 12 bytes of digits per element of A per pass, 21 digit products
    srt = bench._stage_roofline("fp64tc", m, n, l, q, d, prof, 1, peaks)
    assert abs(srt["products_with_A"]["achieved_gbs"] - 4 * 12.0 * m * n / 1e-3 / 1e9) < 1e-6
    assert abs(srt["products_with_A"]["tensor_tflops"] -
               21 * 4 * 2.0 * m * n * l / 1e-3 / 1e12) < 1e-6
    # TF32x3: twice the bytes, half the tensor rate
    sr32 = bench._stage_roofline("tf32x3", m, n, l, q, d, prof, 1, peaks)
    assert abs(sr32["products_with_A"]["achieved_gbs"] - 2 * pa["achieved_gbs"]) < 1e-6
    assert abs(sr32["products_with_A"]["tensor_frac"] - 2 * pa["tensor_frac"]) < 1e-12
    # the FP64 form's products are FP64 flops, without a tensor-core entry
    sr64 = bench._stage_roofline("fp64", m, n, l, q, d, prof, 1, peaks)
    assert sr64["products_with_A"]["bound"] == "alu"
    assert "tensor_frac" not in sr64["products_with_A"]


def test_in_flight_choice():
    sys.path.insert(0, ROOT)
    import bench
    counts = (1, 2, 4, 8)
    sweep = {"direct": {1: 350.0, 2: 500.0, 4: 700.0, 8: 715.0},
             "graph": {1: 380.0, 2: 510.0, 4: 690.0, 8: 700.0}}
    assert bench._pick_in_flight(sweep, counts) == (8, "direct")
    # the faster way at the fastest count, whichever way comes first
    sweep["graph"][8] = 716.0
    assert bench._pick_in_flight(sweep, counts) == (8, "graph")
    # ties go to fewer problems in flight, then to direct calls
    sweep["direct"][4] = 716.0
    assert bench._pick_in_flight(sweep, counts) == (4, "direct")
    sweep["graph"][4] = 716.0
    assert bench._pick_in_flight(sweep, counts) == (4, "direct")
