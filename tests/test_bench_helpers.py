"""bench.py's host-side helpers: the DRAM-traffic figure is reported only
while the kernel sources it was captured on are unchanged (else null), and
the committed summaries name the sources their hash covers."""
import os

import bench


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)


def test_traffic_figure_is_gated_on_the_kernel_sources(tmp_path):
    src = tmp_path / "k.cu"
    _write(src, "__global__ void k() {}\n")
    rel = os.path.relpath(src, bench.ROOT)
    h = bench.kernel_hash([rel])
    tf = tmp_path / "traffic.txt"
    _write(tf, f"# summary\nkernel_sources_sha256_16 = {h}\ndram_bytes_per_page = 21.5\n")
    assert bench.read_traffic(str(tf), [rel], "dram_bytes_per_page") == 21.5
    _write(src, "__global__ void k() { /* changed */ }\n")
    assert bench.read_traffic(str(tf), [rel], "dram_bytes_per_page") is None      # stale: null
    assert bench.read_traffic(str(tmp_path / "missing.txt"), [rel], "dram_bytes_per_page") is None
    _write(tf, f"kernel_sources_sha256_16 = {bench.kernel_hash([rel])}\n")
    assert bench.read_traffic(str(tf), [rel], "dram_bytes_per_page") is None      # no figure: null


def test_committed_traffic_summaries_name_their_sources():
    for path, sources in ((bench.TRAFFIC_FILE, bench.KERNEL_SOURCES),
                          (bench.PROBE_TRAFFIC_FILE, bench.PROBE_SOURCES)):
        text = open(path).read()
        assert "kernel_sources_sha256_16 =" in text
        for s in sources:
            assert os.path.exists(os.path.join(bench.ROOT, s)), s
            assert os.path.basename(s) in text, (path, s)
