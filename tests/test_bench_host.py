"""Host logic of bench.py that needs no GPU: the key that ties the stored ncu traffic of the
evaluator to the code it was captured on, and the JSON fields derived from it."""
import os
import shutil


import bench


def test_strip_comments_keeps_code_and_string_contents():
    src = ('int a = 1; // line comment\n/* block\n comment */ const char* s = "a//b /* c */";\n'
           "char q = '/'; char e = '\\''; int b = a / 2;")
    out = bench._strip_comments(src)
    assert "line comment" not in out and "block" not in out
    assert '"a//b /* c */"' in out
    assert "'/'" in out and "'\\''" in out
    assert "int b = a / 2;" in out


def test_strip_comments_collapses_whitespace():
    assert bench._strip_comments("a  =\n\n\tb ;  // x\n") == bench._strip_comments("a = b ;")


def _copy_sources(tmp_path):
    root = tmp_path / "repo"
    csrc = root / "paper_2311_06952_gb300" / "csrc"
    shutil.copytree(os.path.join(bench.ROOT, "paper_2311_06952_gb300", "csrc"), csrc)
    return str(root), csrc


def test_source_key_ignores_comments_but_not_code(tmp_path, monkeypatch):
    root, csrc = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    base = bench._eval_source_hash()
    hdr = csrc / "eval_kernel.cuh"
    text = hdr.read_text()
    hdr.write_text(text.replace("#pragma once", "// an added comment line\n#pragma once", 1))
    assert bench._eval_source_hash() == base
    hdr.write_text(text.replace("constexpr int kMaxStages = 3;", "constexpr int kMaxStages = 2;", 1))
    assert bench._eval_source_hash() != base


def test_stored_traffic_is_used_only_for_its_code(monkeypatch):
    monkeypatch.setattr(bench, "_eval_source_hash", lambda: bench.EVAL_TRAFFIC["source_sha256_16"])
    assert bench._traffic_default() == bench.EVAL_TRAFFIC["bytes"]
    assert bench._ncu_default() is bench.EVAL_TRAFFIC["ncu"]
    monkeypatch.setattr(bench, "_eval_source_hash", lambda: "0" * 16)
    assert bench._traffic_default() is None
    assert bench._ncu_default() is None


def test_traffic_is_null_for_other_code(tmp_path, monkeypatch):
    root, csrc = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    common = csrc / "common.cuh"
    common.write_text(common.read_text() + "\nnamespace deoct { constexpr int kChanged = 1; }\n")
    assert bench._traffic_default() is None
    assert bench._ncu_default() is None


def test_source_key_covers_the_device_helpers_only(tmp_path, monkeypatch):
    """common.cuh's host-side context and error codes are not the kernel's code; its device
    helpers are."""
    root, csrc = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    base = bench._eval_source_hash()
    common = csrc / "common.cuh"
    text = common.read_text()
    common.write_text(text.replace("  int device = 0;", "  int device = 0;\n  int unrelated_host_field = 0;", 1))
    assert bench._eval_source_hash() == base
    common.write_text(text.replace("return (uint32_t)(((uint64_t)x * (uint64_t)m) >> 32);",
                                   "return (uint32_t)(((uint64_t)x * (uint64_t)m) >> 31);", 1))
    assert bench._eval_source_hash() != base


def test_source_key_covers_the_shape_chooser(tmp_path, monkeypatch):
    """The stored counters belong to one launch shape: a change of the chooser's constants
    changes the key."""
    root, csrc = _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    base = bench._eval_source_hash()
    ev = csrc / "eval.cu"
    text = ev.read_text()
    assert "25000.0 + 170.0 * copies" in text
    ev.write_text(text.replace("25000.0 + 170.0 * copies", "26000.0 + 170.0 * copies", 1))
    assert bench._eval_source_hash() != base


def test_reference_arm_prints_one_line_with_the_contract_keys():
    """`bench.py --impl reference` (the oracle on the host's cores, no GPU) prints one JSON
    line on the main arm's metric, unit and direction, with its CPU baseline and an
    end-to-end entry that copies nothing."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="0")
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, cwd=root, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
