"""The algorithmic amounts that bench.py divides by measured times for its
roofline figures, worked out by hand for the 5M-observation scene (1,800
cameras, 1,000,000 landmarks, 4,999,149 observations), and the traffic
lookup's refusal of stale or unknown keys (no GPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

N_OBS, N_PTS = 4_999_149, 1_000_000


def test_series_bytes_per_product():
    # 12 B per observation (u32 camera + f32x2 measurement), 40 B per landmark
    assert bench.series_bytes_per_term(N_OBS, N_PTS) == 59_989_788 + 40_000_000
    # stored schedule: the camera index and the stored block replace the measurement
    assert bench.series_bytes_per_term(N_OBS, N_PTS, 36) == 40 * N_OBS + 40 * N_PTS
    assert bench.series_bytes_per_term(N_OBS, N_PTS, 18) == 22 * N_OBS + 40 * N_PTS
    assert bench.block_build_bytes(N_OBS, 36) == 48 * N_OBS


def test_landmark_work_per_launch():
    assert bench.landmark_df_ops_per_launch(N_OBS, N_PTS) == 635 * N_OBS + 400 * N_PTS
    assert bench.landmark_flops_per_launch(N_OBS, N_PTS) == 98 * N_OBS + 60 * N_PTS


def test_traffic_lookup_refuses_unknown_keys_and_sources():
    assert bench.ncu_traffic("series.cu", "no_such_kernel") is None
    assert bench.ncu_traffic("no_such_file.cu", "series_product_s1") is None


def test_code_hash_ignores_comments_but_not_code(tmp_path):
    base = "int f(int a) {\n  return a + 1;  // one more\n}\n"
    p = tmp_path / "k.cu"
    p.write_text(base)
    h = bench.code_hash(str(p))
    p.write_text("/* a kernel\n   note */\nint f(int a) {\n\n    return a + 1;   // another note\n}\n")
    assert bench.code_hash(str(p)) == h          # comments, blank lines, indentation
    p.write_text(base.replace("a + 1", "a + 2"))
    assert bench.code_hash(str(p)) != h          # a change of code
