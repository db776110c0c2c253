"""Host logic of bench.py (no GPU): the algorithmic-byte model, the rooflines built from
measured peaks, and the profile summaries it reads (only when their kernel-source digest is
the current one)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_pass_bytes_counts_the_schedule():
    """Forward: one P2G, T-1 fused passes (full state at checkpoints and over the resident
    last segment), one last G2P; backward: per re-simulated segment one P2G, its fused
    passes and one G2P; one adjoint pass per step."""
    N, T, K, d = 1000, 24, 8, 3
    a = bench.alg_bytes(d)
    by = bench.pass_bytes(N, T, K, d, kept=True)
    sL = ((T - 1) // K) * K  # 16: the resident last segment starts here
    n_full_fwd = sum(1 for t in range(1, T) if t % K == 0 or t > sL)
    n_resim = sum(min(K, T - s0) - 1 for s0 in range(0, sL, K))
    assert by["g2p_p2g"] == (T - 1 - n_full_fwd) * a["g2p_p2g"] * N
    assert by["g2p_p2g_full"] == (n_full_fwd + n_resim) * a["g2p_p2g_full"] * N
    # recomputing the grids costs bytes, keeping them does not
    assert bench.pass_bytes(N, T, K, d, kept=False)["adj_fused"] > by["adj_fused"]


def test_scatter_roofline_from_measured_peaks():
    class FakeMPM:
        MPM_PEAK_RED_F32X4, MPM_PEAK_RED_F32X4_SPREAD = 2, 3

        @staticmethod
        def mpm_measure_peak(kind):
            return {2: 4.0e11, 3: 2.0e11}[kind]

    # 10 launches of 1 ms each over 1,000 particles of a 3D scene: 27e3 reductions a launch
    prof = {"g2p_p2g": (10, 10.0), "adj_fused": (5, 10.0), "g2p": (1, 1.0)}
    r = bench.scatter_roofline(FakeMPM, prof, 1000, 3)
    assert r["reductions_per_particle"] == 27 and r["peak"] == 4.0e11
    g = r["kernels"]["g2p_p2g"]
    assert g["achieved"] == pytest.approx(27e3 / 1e-3)
    assert g["frac"] == pytest.approx(27e6 / 4.0e11) and g["frac_spread"] == pytest.approx(27e6 / 2.0e11)
    assert r["kernels"]["adj_fused"]["avg_launch_ms"] == pytest.approx(2.0)
    assert "g2p" not in r["kernels"]  # the last G2P scatters nothing


def test_profiles_are_read_only_on_their_digest(tmp_path, monkeypatch):
    """A committed summary carrying the current digest is read; one with another digest, or
    none, gives None (the bench then reports null rather than stale counters)."""
    digest = bench.source_digest()
    prof_dir = tmp_path / "profiles"
    prof_dir.mkdir()
    (prof_dir / "ncu_adj_fused_w.md").write_text(
        f"source digest: {digest}\n\n| `dram__bytes_read.sum` | 2.0 | 4.0 | Mbyte |\n"
        "| `dram__bytes_write.sum` | 1.0 | 1.0 | Kbyte |\n")
    (prof_dir / "fp64_adj_fused_w.md").write_text(
        f"source digest: {digest}\nFP64 FLOP per particle: 0.0\nFP32 FLOP per particle: 4400\n")
    (prof_dir / "ncu_adj_fused_old.md").write_text(
        "source digest: 0000000000000000\n| `dram__bytes_read.sum` | 2.0 | Mbyte |\n"
        "| `dram__bytes_write.sum` | 1.0 | Mbyte |\n")
    monkeypatch.setattr(bench, "source_digest", lambda: digest)  # of the real sources
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("w", "adj_fused") == pytest.approx(3.0e6 + 1.0e3)
    assert bench.flop_per_particle("w", "adj_fused") == 0.0
    assert bench.flop_per_particle("w", "adj_fused", "FP32") == 4400.0
    assert bench.profiled_traffic("old", "adj_fused") is None
    assert bench.profiled_traffic("none", "adj_fused") is None
