"""Host-side parts of bench.py that need no GPU: the host description and
copy rate reported beside the oracle's time."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_host_info_reports_model_and_copy_rate():
    import bench
    info = bench.host_info(n_doubles=1 << 20, reps=2)
    assert isinstance(info["cpu_model"], str) and info["cpu_model"]
    assert info["host_copy_gbs"] > 0
    assert info["host_copy_threads"] == (os.cpu_count() or 1)
