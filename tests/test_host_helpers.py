"""Host-side helpers that need no GPU: the benchmark's profiled-traffic reader and the surrogate
driver's input normalisation, error metric and resumable sample file."""
import json

import numpy as np
import pytest


def test_profiled_traffic_reads_the_committed_summary():
    import bench
    t = bench.profiled_traffic("k_spmv_f32<8>", 4932870)
    assert t is not None and t > 0
    # scaling is linear in the number of blocks
    assert bench.profiled_traffic("k_spmv_f32<8>", 2 * 4932870) == pytest.approx(2 * t)
    assert bench.profiled_traffic("no_such_kernel", 10) is None


def test_job_rate_and_positions():
    import bench
    z = bench.probe_positions(4, 0, 1)
    assert np.allclose(np.diff(z), 0.5e-3) and z.size == 4
    assert bench.job_rate(16, 1, 4.0) == 4.0


def test_surrogate_input_normalisation_maps_ranges_to_unit_box():
    from paper_1602_03207_gb300 import surrogate as S
    lo = S.normalise_inputs(S.LO)
    hi = S.normalise_inputs(S.HI)
    mid = S.normalise_inputs(0.5 * (S.LO + S.HI))
    assert np.allclose(lo, -1.0) and np.allclose(hi, 1.0) and np.allclose(mid, 0.0, atol=1e-7)
    assert lo.dtype == np.float32


def test_relative_errors_per_row():
    from paper_1602_03207_gb300 import surrogate as S
    ref = np.array([[3.0, 4.0], [1.0, 0.0]])
    pred = np.array([[3.0, 4.0], [0.0, 0.0]])
    assert np.allclose(S.relative_errors(pred, ref), [0.0, 1.0])


def test_sample_file_resume_skips_cut_lines(tmp_path):
    from paper_1602_03207_gb300 import surrogate as S
    path = tmp_path / "s.jsonl"
    recs = [{"seed": s, "params": [0.0] * 6, "dz_re": [1.0], "dz_im": [0.0]} for s in (3, 1)]
    with open(path, "w") as f:
        for r in recs:
            f.write(json.dumps(r) + "\n")
        f.write('{"seed": 7, "params": [0.0')                 # a line cut by an interruption
    got = S.load_samples(str(path))
    assert sorted(got) == [1, 3]
    X, Y = S.arrays(got, [1, 3])
    assert X.shape == (2, 6) and Y.shape == (2, 2)
    assert S.load_samples(str(tmp_path / "missing.jsonl")) == {}
