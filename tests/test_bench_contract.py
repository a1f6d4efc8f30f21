"""CPU checks of bench.py's host logic: the reference arm's JSON line (the FP64 oracle timed
on a bounded sample) and the per-kernel work model behind the roofline."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "it/s" and d["steps"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "1080x1920-C3-L3-N200k"
    # both arms print the same config object for the same run
    import bench
    from paper_2511_15022_gb300 import inputs
    assert d["config"] == json.loads(json.dumps(bench.workload_config(inputs.hd_1080p(),
                                                                       "autograd", 1)))
    small = d["small_workload_full_steps"]
    assert small["workload"] == "small-256x256-C1-L1-N2048" and small["s_per_step"] > 0


def test_work_model_matches_the_fused_pass_count():
    """Fused step: 12 + 8.5 L units of S = H W 8 bytes per channel over the FFT passes and
    raster field accesses; the autograd step adds a forward-only pass (1 + 3 + (2 + 2L) +
    2.5 L units)."""
    import bench
    from paper_2511_15022_gb300 import inputs
    w = inputs.hd_1080p()
    S = w.H * w.W * 8
    fused = bench.step_work(w, "fused", pairs=0.0)
    auto = bench.step_work(w, "autograd", pairs=0.0)
    field = {"k_rows_pad_fwd", "k_cols_fwd_planes", "k_rows_loss", "k_cols_bwd_planes",
             "k_rows_inv_crop"}
    units_fused = sum(v[0] for k, v in fused.items() if k in field) / (w.C * S)
    units_fused += 2  # raster field write + read (the records are per Gaussian, not per pixel)
    assert abs(units_fused - (12 + 8.5 * w.L)) < 1e-9
    units_auto = sum(v[0] for k, v in auto.items() if k in field) / (w.C * S) + 3
    assert abs(units_auto - (12 + 8.5 * w.L + 1 + 3 + 2 + 2 * w.L + 2.5 * w.L)) < 1e-9
    assert auto["k_cols_fwd_planes"][3] == 2 and fused["k_cols_fwd_planes"][3] == 1


def test_work_model_with_an_identity_plane():
    """With the plane at 0 mm taken in the pixel domain the column and loss-row passes count
    the two propagated planes only, and the forward raster reads one target plane and writes
    the seed, which the last row pass reads back."""
    import bench
    from paper_2511_15022_gb300 import inputs
    w = inputs.hd_1080p()
    S = w.H * w.W * 8
    full = bench.step_work(w, "fused", pairs=0.0)
    ident = bench.step_work(w, "fused", pairs=0.0, ident=1)
    assert ident["k_cols_fwd_planes"][0] == (2 + 2 * 2) * w.C * S
    assert ident["k_cols_bwd_planes"][0] == (2 * 2 + 2) * w.C * S
    assert ident["k_rows_loss"][0] == 4.5 * 2 * w.C * S
    assert ident["k_raster_fwd"][0] == full["k_raster_fwd"][0] + 1.5 * w.C * S
    assert "k_ident_loss" not in ident
    assert ident["k_rows_inv_crop"][0] == full["k_rows_inv_crop"][0] + w.C * S
    # one column transform of the four per column block fewer in each column pass
    assert abs(ident["k_cols_fwd_planes"][1] / full["k_cols_fwd_planes"][1] - 3 / 4) < 0.01
    assert bench.algorithmic_bytes(w, 1)["k_cols_fwd_planes"] == ident["k_cols_fwd_planes"][0]
