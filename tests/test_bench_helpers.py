"""Host-side checks of bench.py's bookkeeping (no GPU): the committed Nsight Compute figures are
well-formed and name profiled kernels whose sources exist, and the lookup keys them by the
kernel's own sources."""
import glob
import os

import bench

PROFILES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")


def _figure_lines():
    out = []
    for f in glob.glob(os.path.join(PROFILES, "*.md")) + glob.glob(os.path.join(PROFILES, "*.txt")):
        for line in open(f):
            if line.startswith(("TRAFFIC ", "INST ")):
                out.append((os.path.basename(f), line.split()))
    return out


def test_profile_figures_are_well_formed():
    lines = _figure_lines()
    assert lines, "no TRAFFIC/INST lines under profiles/"
    for fname, toks in lines:
        kv = dict(t.split("=", 1) for t in toks[1:])
        assert kv["kernel"] in bench.KERNEL_SOURCES, (fname, kv)
        assert len(kv["src_sha"]) == 16 and int(kv["src_sha"], 16) >= 0, (fname, kv)
        vals = [v for k, v in kv.items() if k not in ("kernel", "src_sha")]
        assert len(vals) == 1 and float(vals[0]) > 0, (fname, kv)


def test_kernel_sources_exist_and_hash():
    for kernel, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(bench.ROOT, "paper_1306_6291_gb300", "csrc", f)), f
        sha = bench.kernel_sha(kernel)
        assert len(sha) == 16 and sha == bench.kernel_sha(kernel)


def test_lookup_ignores_figures_of_other_sources(monkeypatch):
    """A figure counts only for the sources it was taken on."""
    monkeypatch.setattr(bench, "kernel_sha", lambda kernel: "0" * 16)
    assert bench.profile_figure("TRAFFIC", "k_eig3_adj", "bytes_per_matrix") is None
    assert bench.traffic_for("k_eig3_adj", 1 << 24) is None
