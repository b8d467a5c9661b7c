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


def test_algorithmic_bytes_follow_the_per_row_table():
    """Per row: 34 B per residual evaluation (+ the residual's matrix bytes),
    18 B per update, 20 B + one H application per CG iteration, 26 B + two S
    applications per CGNR iteration; applications of 4 B (constant stencil),
    10 B for H with face coefficients, 7 x (2 + 4) + 4 + 4 = 50 B for FP16 CSR
    (104 B in FP64)."""
    import bench
    info = {"outer_iters": 2, "inner_iters_H": 3, "inner_iters_S": 4}
    n = 1000
    assert bench.algorithmic_bytes(n, 7 * n, info, "stencil") == n * (3 * 34 + 2 * 18 + 3 * 24 + 4 * 34)
    faces = 3 * (34 + 24) + 2 * 18 + 3 * (20 + 10) + 4 * (26 + 2 * 4)
    assert bench.algorithmic_bytes(n, 7 * n, info, "stencil", faces=True) == n * faces
    csr = 3 * (34 + 7 * 12 + 4) + 2 * 18 + 3 * (20 + 50) + 4 * (26 + 2 * 50)
    assert bench.algorithmic_bytes(n, 7 * n, info, "sparse") == n * csr
    assert bench.spmv_bytes("sparse", False) == 104 and bench.spmv_bytes("stencil", False) == 16
    assert bench.spmv_bytes("stencil", False, faces=True, op="H") == 40
    fp64 = 3 * 34 + 2 * 18 + 3 * (80 + 16) + 4 * (104 + 32)
    assert bench.algorithmic_bytes(n, 7 * n, info, "stencil", fp16=False) == n * fp64


def test_profiled_traffic_needs_the_current_sources(tmp_path, monkeypatch):
    """The DRAM bytes of a committed capture are scaled by algorithmic bytes,
    and dropped (None) once the kernel's sources differ from the capture's."""
    import bench
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_2501_04229_gb300").symlink_to(os.path.join(bench.ROOT, "paper_2501_04229_gb300"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.kernel_source_digest()
    f = tmp_path / "profiles" / "k.md"
    f.write_text(f"# k\n\nkernel-source-sha256: {digest}\ndram-bytes-per-launch: 500\n"
                 "algorithmic-bytes-per-launch: 1000\n")
    assert bench.profiled_traffic("k.md", 3000) == 1500
    f.write_text("kernel-source-sha256: 0000000000000000\ndram-bytes-per-launch: 500\n"
                 "algorithmic-bytes-per-launch: 1000\n")
    assert bench.profiled_traffic("k.md", 3000) is None
    assert bench.profiled_traffic("missing.md", 3000) is None


def test_solve_kernel_name_follows_the_info():
    import bench
    assert bench.solve_kernel_name("sparse", {"zmarch_planes": 0}) == "gadi_solve_kernel<EllOp<half>>"
    assert bench.solve_kernel_name("stencil", {"zmarch_planes": 12}).startswith("gadi_solve_kernel<ZMarchOp<")
    assert bench.solve_kernel_name("stencil", {"zmarch_planes": 0}) == "gadi_solve_kernel<StencilOp<half,3,8>>"
