"""CPU checks of the benchmark's bookkeeping: committed ncu traffic records are used only while
the code they were taken from is unchanged (comments aside), and the harmonic-sum defaults."""
import importlib.util
import json
import os
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_code_only_drops_comments_not_strings():
    b = _bench()
    a = 'int x = 1; // note\n/* block\n comment */ const char *s = "a // b /* c */";\n'
    c = 'int x = 1;\nconst char *s = "a // b /* c */"; // other note\n'
    assert b._code_only(a) == b._code_only(c)
    assert '"a // b /* c */"' in b._code_only(a)
    assert b._code_only("int x = 1;") != b._code_only("int x = 2;")


def _fake_tree(tmp_path, b, kind):
    csrc = tmp_path / "paper_1805_12280_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in b.KERNEL_SOURCES[kind]:
        shutil.copy(os.path.join(ROOT, "paper_1805_12280_gb300", "csrc", fn), csrc / fn)
    (tmp_path / "profiles").mkdir()
    return csrc


@pytest.mark.parametrize("kind,record", [("fp32", "ols_fp32_L2048_n2p22_traffic.json"),
                                         ("harmonic", "harmonic_sum_h8_n2p22_traffic.json")])
def test_traffic_record_follows_the_code(tmp_path, monkeypatch, kind, record):
    b = _bench()
    csrc = _fake_tree(tmp_path, b, kind)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    rec = {"dram_bytes_per_launch": 123456, "kernel_sources_sha256": b.kernel_sources_sha256(kind)}
    (tmp_path / "profiles" / record).write_text(json.dumps(rec))
    get = (lambda: b.profile_traffic("fp32")) if kind == "fp32" else (lambda: b.profile_traffic(kind, record))
    assert get() == 123456
    first = b.KERNEL_SOURCES[kind][0]
    src = (csrc / first).read_text()
    (csrc / first).write_text(src + "\n// a comment changes nothing\n")
    assert get() == 123456
    (csrc / first).write_text(src + "\nstatic int added_code = 1;\n")
    assert get() is None                     # the record no longer describes this code


def test_committed_records_name_their_workload():
    for fn in ("ols_fp32_L2048_n2p22_traffic.json", "ols_tc_L2048_n2p22_traffic.json",
               "harmonic_sum_h8_n2p22_traffic.json"):
        with open(os.path.join(ROOT, "profiles", fn)) as f:
            d = json.load(f)
        assert d["dram_bytes_read"] + d["dram_bytes_write"] == d["dram_bytes_per_launch"]
        assert "2^22" in d["workload"] and d["command"].startswith("ncu ")
        assert "--clock-control none" in d["command"]


def test_harmonic_defaults():
    import paper_1805_12280_gb300 as fd
    assert fd.harmonic_levels(1) == [1] and fd.harmonic_levels(32) == [1, 2, 4, 8, 16, 32]
    thr = fd.harmonic_thresholds(8)
    assert thr[0] == 7.0 and thr[2] == 16.0 and thr[3] == pytest.approx(8 + 6 * 8 ** 0.5)


def test_oracle_harmonic_timing_record():
    b = _bench()
    rec = b.time_oracle_harmonic(85, 1 << 16, 210, 8, [7.0, 10.49, 16.0, 24.97], cols=1 << 13)
    assert rec["kind"] == "oracle" and rec["unit"] == "arrays/s" and rec["cores"] >= 1
    assert rec["value"] > 0 and "85 x 8192" in rec["sample"]
