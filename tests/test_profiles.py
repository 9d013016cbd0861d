"""The committed ncu summaries under profiles/ are what bench.py reports as
`roofline.traffic`: each must give its command, numeric per-launch traffic
for the three finest-level passes and the SHA-256 of the kernel sources the
counters were taken on, and contain no unfilled template text.  (Whether the
hash still matches the sources is bench.py's business: a stale summary makes
it report traffic as null, it is not an error.)"""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def summaries():
    d = os.path.join(ROOT, "profiles")
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith(".md"))


def test_every_summary_is_filled_in_and_names_its_command():
    paths = summaries()
    assert paths
    for p in paths:
        txt = open(p).read()
        assert re.search(r"\{[a-z_][a-z0-9_]*(\[[^\]]*\])?[^}]*\}", txt) is None, f"template text left in {p}"
        assert "ncu " in txt and "--clock-control none" in txt, p
        assert re.search(r"^source_sha256: [0-9a-f]{64}$", txt, flags=re.M), p


def test_bench_reads_traffic_for_the_three_passes():
    b = load_bench()
    keys = {b.PROFILE_SUMMARY: ("spmv_pq", "resid", "up0"), b.STREAM_SUMMARY: ("pq", "resid", "up0")}
    for path, want in keys.items():
        txt = open(path).read()
        got = dict(re.findall(r"traffic_bytes_per_launch\[(\w+)\]:\s*([0-9.eE+]+)", txt))
        assert set(want) <= set(got), (path, got)
        for k in want:
            # a full 3-D p=3 n=64 launch moves hundreds of MB
            assert 1e8 < float(got[k]) < 2e9, (path, k, got[k])


def test_a_stale_summary_reports_no_traffic(tmp_path):
    """bench.py takes traffic from a summary only while the recorded SHA-256
    matches the current kernel sources; otherwise it reports null."""
    import hashlib

    b = load_bench()
    src = ("sell_kernels.cu",)
    h = hashlib.sha256(open(os.path.join(ROOT, "paper_2511_21268_gb300", "csrc", src[0]), "rb").read()).hexdigest()
    body = "traffic_bytes_per_launch[pq]: 123456789\n"
    good = tmp_path / "good.md"
    good.write_text(body + f"source_sha256: {h}\n")
    stale = tmp_path / "stale.md"
    stale.write_text(body + "source_sha256: " + "0" * 64 + "\n")
    assert b.committed_traffic(str(good), src) == {"pq": 123456789.0}
    assert b.committed_traffic(str(stale), src) is None
    assert b.committed_traffic(str(tmp_path / "missing.md"), src) is None
