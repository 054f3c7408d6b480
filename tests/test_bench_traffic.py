"""The bench's roofline `traffic` comes from a committed ncu summary only
while the CUDA sources are the ones the counters were taken on (CPU)."""
import bench


def test_committed_traffic_follows_the_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "csrc"
    csrc.mkdir()
    (csrc / "k.cu").write_text("kernel v1\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "CSRC", str(csrc))
    monkeypatch.setattr(bench, "PROFILES", str(prof))
    sha = bench.sources_sha()
    (prof / "k_wl.md").write_text("# summary\n\n`traffic wl per-iteration 2359 sources %s`\n" % sha)
    assert bench.committed_traffic("wl", "per-iteration") == (2359.0, "k_wl.md")
    # another workload or unit: no figure
    assert bench.committed_traffic("other", "per-iteration")[0] is None
    assert bench.committed_traffic("wl", "per-launch")[0] is None
    # a kernel source changed after the capture: the figure no longer applies
    (csrc / "k.cu").write_text("kernel v2\n")
    value, why = bench.committed_traffic("wl", "per-iteration")
    assert value is None and "changed" in why


def test_committed_profiles_parse():
    # every traffic line committed under profiles/ has the parsed form
    import glob
    import os
    import re
    pat = re.compile(r"^traffic\s+(\S+)\s+(\S+)\s+([0-9.eE+]+)\s+sources\s+([0-9a-f]{16})$")
    lines = []
    for f in glob.glob(os.path.join(bench.PROFILES, "*.md")):
        with open(f) as fh:
            lines += [ln.strip().strip("`") for ln in fh if ln.strip().strip("`").startswith("traffic ")]
    assert lines
    for ln in lines:
        assert pat.match(ln), ln
