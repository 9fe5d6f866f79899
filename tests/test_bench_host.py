"""Host helpers of bench.py (no GPU): the roofline's HBM peak comes from the
measured peaks file when it is present and from the stated fallback when not;
the FP64 peak is the derived FP64-pipe figure; the QR flop count reduces to
4/3 n^3 for a square matrix."""
import json
import os

import bench


def test_hbm_peak_from_file_and_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 1234.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench.hbm_peak_gbs()
    assert peak == 1234.5 and "MEASURED_PEAKS.json" in src
    os.remove(tmp_path / "MEASURED_PEAKS.json")
    peak, src = bench.hbm_peak_gbs()
    assert peak == 6800.0 and src.startswith("fallback")


def test_fp64_peak_and_qr_flops():
    assert abs(bench.FP64_PEAK_TFLOPS - 1.25856) < 1e-9
    n = 16384
    assert abs(bench.flops_qr(n, n) / (4.0 * n ** 3 / 3.0) - 1.0) < 1e-14
    assert abs(bench.flops_qr(300, 200) / (2.0 * 300 * 200 ** 2 - 2.0 * 200 ** 3 / 3.0) - 1.0) < 1e-14


def test_cpu_context_times_the_oracle_and_lapack():
    out = bench.cpu_context(m=200, n=120, k=8, b=4, p=4, nq=64)
    assert out["cores"] >= 1
    for key in ("oracle_tuxv_200x120_k8_s", "lapack_dgeqrf_64_s", "lapack_dgeqp3_64_s"):
        assert out[key] > 0.0


def test_trailing_counts():
    """The trailing update touches sum_J m_t n2 entries (about n^3 / (3 b) for a
    square matrix), and its tensor-core flops are 36 slice pairs of the two
    2 m_t n2 b_J products."""
    import bench
    n, b = 4096, 64
    ent = bench.trailing_entries(n, n, b)
    assert abs(ent / (n ** 3 / (3 * b)) - 1) < 0.03
    assert bench.trailing_entries(100, 50, 64) == 100 * (50 - 50)  # one block covers every column
    fl = bench.slice_pair_flops(n, n, b)
    assert abs(fl - 36 * 4 * b * ent) / fl < 1e-12
