"""Host logic of bench.py that needs no GPU: the source hash that keeps or drops the committed
ncu traffic figure, and the lookup of that figure."""
import os
import shutil

import bench


def _copy_sources(tmp_path):
    root = tmp_path / "repo"
    csrc = root / "paper_1006_0549_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, "paper_1006_0549_gb300", "csrc", f), csrc / f)
    return root, csrc


def test_source_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    root, csrc = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.kernel_source_hash()
    f = csrc / "lpdf_pipeline.cu"
    text = f.read_text()
    f.write_text("// an added line comment\n/* and a\n block comment */\n\n" + text.replace("\n", "\n\n", 3))
    assert bench.kernel_source_hash() == h0
    f.write_text(text.replace("constexpr int kLaneChunk = 8;", "constexpr int kLaneChunk = 4;"))
    assert bench.kernel_source_hash() != h0


def test_traffic_figure_follows_the_hash(tmp_path, monkeypatch):
    root, csrc = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    prof = tmp_path / "traffic.txt"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(prof))
    prof.write_text("variant 2 bytes per particle: 77.5\nkernel_source_hash: %s\n" % bench.kernel_source_hash())
    assert bench.ncu_traffic(1000, 2) == 77500.0
    assert bench.ncu_traffic(1000, 3) is None          # no figure for that variant
    (csrc / "lpdf_device.cuh").write_text((csrc / "lpdf_device.cuh").read_text() + "\nnamespace lpdf {}\n")
    assert bench.ncu_traffic(1000, 2) is None          # taken on other code


def test_aux_section_records_library_errors_and_raises_the_rest():
    from paper_1006_0549_gb300 import lpdf

    def lost():
        raise lpdf.LpdfError(lpdf.LPDF_ERR_LOST_PARTICLE, "3 particle(s) lost")

    def bug():
        raise ValueError("not a library status")

    assert bench.aux_section(lambda a, b=1: {"v": a + b}, 2, b=3) == {"v": 5}
    assert "lost" in bench.aux_section(lost)["error"]
    try:
        bench.aux_section(bug)
    except ValueError:
        pass
    else:
        raise AssertionError("a non-library error must propagate")


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores, on a bounded sample of the
    channel workload) prints one JSON line with the fields of the bench contract."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] >= 3
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "particle-updates/s"
    assert d["metric"].startswith("particle-updates/s")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "channel-50k-25M"
