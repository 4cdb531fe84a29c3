"""The benchmark's guard on measured figures: a per-event FP64 count or a
DRAM traffic figure is used only while the transport kernels' sources are
the ones it was measured on (their digest); any edit of those sources marks
it stale.  CPU only."""
import os
import shutil

import bench


def test_digest_covers_every_transport_source_and_changes_with_any_edit(tmp_path):
    src = os.path.join(bench.ROOT, "paper_2506_00263_gb300", "csrc")
    for name in bench.TRANSPORT_SOURCES:
        assert os.path.exists(os.path.join(src, name)), name
    copy = tmp_path / "csrc"
    shutil.copytree(src, copy)
    d0 = bench.kernel_digest(str(copy))
    assert d0 == bench.kernel_digest(src) and len(d0) == 16
    for name in bench.TRANSPORT_SOURCES:
        p = copy / name
        text = p.read_text()
        p.write_text(text + "\n// an edit\n")
        assert bench.kernel_digest(str(copy)) != d0, name
        p.write_text(text)
    assert bench.kernel_digest(str(copy)) == d0
    # files outside the transport kernels do not enter the digest
    (copy / "tr_capi.cu").write_text((copy / "tr_capi.cu").read_text() + "\n// host code\n")
    assert bench.kernel_digest(str(copy)) == d0


def test_measured_figures_are_fresh_only_on_their_digest(monkeypatch):
    table = {"k": (12.5, "0123456789abcdef")}
    monkeypatch.setattr(bench, "kernel_digest", lambda csrc=None: "0123456789abcdef")
    assert bench.measured_figure(table, "k") == (12.5, True)
    monkeypatch.setattr(bench, "kernel_digest", lambda csrc=None: "fedcba9876543210")
    assert bench.measured_figure(table, "k") == (12.5, False)
    assert bench.measured_figure(table, "missing") == (None, False)
    # the stored figures name a digest of the same form
    for tab in (bench.FP64_OPS, bench.TRAFFIC):
        for value, digest in tab.values():
            assert value > 0 and len(digest) == 16 and int(digest, 16) >= 0
