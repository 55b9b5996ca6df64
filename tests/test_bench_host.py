"""Host-side logic of bench.py (no GPU): the key that ties a measured DRAM-traffic record to
the sweep kernels' code, the record lookup, and the roofline entry's choice of bound."""
import os

import numpy as np
import pytest

import bench


def test_sweep_code_digest_ignores_comments_and_whitespace():
    a = bench.sweep_code_digest(["int a = 1;  // one\n", "/* block\n comment */ float b;\n"])
    b = bench.sweep_code_digest(["int a = 1;\n\n", "  float   b;"])
    assert a == b
    assert bench.sweep_code_digest(["int a = 2;", "float b;"]) != a   # a code change is seen


def _tree(tmp_path, code, records):
    csrc = tmp_path / "paper_2111_13483_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "ops.cu").write_text(code)
    (csrc / "tile.cuh").write_text("// tile\nint t;\n")
    (csrc / "cluster.cuh").write_text("// cluster\nint u;\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.md").write_text("# summary\n\n" + "\n".join(records) + "\n")


def test_traffic_record_lookup(tmp_path, monkeypatch):
    code = "__global__ void k() {}\n"
    digest = bench.sweep_code_digest([code, "// tile\nint t;\n", "// cluster\nint u;\n"])
    _tree(tmp_path, code, [
        "traffic-record: class=sweep_fwd workload=sphere30720 precision=1 columns=64 bytes=123 source=%s" % digest,
        "traffic-record: class=sweep_bwd workload=sphere30720 precision=1 columns=64 bytes=456 source=0000",
        "traffic-record: class=sweep_fwd workload=sphere7680 precision=0 columns=16 ratio=1.25 source=%s" % digest,
    ])
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.traffic_record("sweep_fwd", "sphere30720", 1)
    assert got is not None and got[0] == 123 and got[2] == 64 and got[3] == os.path.join("profiles", "k.md")
    assert bench.traffic_record("sweep_bwd", "sphere30720", 1) is None      # taken on other code
    assert bench.traffic_record("sweep_fwd", "plate29800", 1) is None       # bytes of another workload
    # a ratio measured on a smaller case serves any workload of the same kernel and precision
    got = bench.traffic_record("sweep_fwd", "sphere30720", 0)
    assert got[0] is None and got[1] == 1.25 and got[2] == 16 and got[4] == "sphere7680"
    # a comment edit of the kernel source keeps the record valid
    (tmp_path / "paper_2111_13483_gb300" / "csrc" / "ops.cu").write_text("// edited\n" + code)
    assert bench.traffic_record("sweep_fwd", "sphere30720", 1)[0] == 123


@pytest.mark.parametrize("cols", [64 * 10, 1 * 10])
def test_sweep_roofline_is_against_hbm(cols):
    # ten complex-FP32 sweep launches over 1e6 stored coefficient entries (of 1.5e6 dense); n = 1000:
    # the solve's operator is reported against HBM at any width, with the ALU figures beside it
    nnzL, n, launches = 1_000_000, 1000, 10
    prof = {"sweep_fwd": (launches, launches, 20.0, cols), "dots": (5, 5, 1.0, 5)}
    fs = {"nnzL": 1_500_000, "update_flops": 1.0, "update_launches": 1}
    cls, r = bench.roofline(prof, fs, {"far_entries": 0, "coef_entries": nnzL}, n, 1)
    assert cls == "sweep_fwd" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    flops = 8.0 * nnzL * cols
    bytes_ = 8.0 * (nnzL * launches + 2.0 * n * cols)
    assert r["intensity_flop_per_byte"] == pytest.approx(flops / bytes_)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["achieved"] == pytest.approx(bytes_ / 0.020 / 1e9)
    assert r["alu_achieved_tflops"] == pytest.approx(flops / 0.020 / 1e12)
    assert r["alu_frac"] == pytest.approx(r["alu_achieved_tflops"] / r["alu_peak_tflops"])


@pytest.mark.parametrize("flops_per_byte, bound", [(100.0, "alu"), (0.5, "hbm")])
def test_setup_roofline_bound_follows_intensity(flops_per_byte, bound):
    # Schur updates: the bound is the one the intensity selects against the ridge
    n, launches = 1000, 4
    nnzL = 1_000_000
    fs = {"nnzL": nnzL, "update_flops": flops_per_byte * 8.0 * nnzL * 3.0, "update_launches": launches}
    prof = {"update": (launches, launches, 10.0, 0), "dots": (1, 1, 0.1, 1)}
    cls, r = bench.roofline(prof, fs, {"far_entries": 0, "coef_entries": nnzL}, n, 1)
    assert cls == "update" and r["bound"] == bound
    assert r["intensity_flop_per_byte"] == pytest.approx(flops_per_byte)


def test_random_rhs_directions_and_polarisations():
    """--rhs random: unit propagation directions spread over the whole sphere, each wave
    polarised perpendicular to its direction, reproducible from the seed."""
    class Rec:
        def __init__(self):
            self.calls = []

        def plane_wave(self, khat, pol):
            self.calls.append((np.array(khat), np.array(pol)))
            return np.zeros(3, np.complex128)
    a, b = Rec(), Rec()
    bench.rhs_batch(a, 512, mode="random")
    bench.rhs_batch(b, 512, mode="random")
    K = np.array([c[0] for c in a.calls])
    Pp = np.array([c[1] for c in a.calls])
    assert np.allclose(np.linalg.norm(K, axis=1), 1.0) and np.allclose(np.linalg.norm(Pp, axis=1), 1.0)
    assert np.max(np.abs(np.sum(K * Pp, axis=1))) < 1e-12
    assert abs(np.mean(K[:, 2])) < 0.1 and K[:, 2].min() < -0.9 and K[:, 2].max() > 0.9
    assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) for x, y in zip(a.calls, b.calls))
