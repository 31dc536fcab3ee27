"""Host-side pieces of bench.py that need no GPU: the gather-aware bound and
the ingestion of an ncu CSV into the traffic record."""
import json

import bench


def test_gather_aware_bound_limits():
    m = k = 1000
    nnz, n, peak = 16_000, 64, 1000.0  # GB/s
    ms = {n: 1.0}
    # all gathers hit L2 (tiny B): the bound is A + C only
    g = bench.gather_aware("none", "other", m, nnz, k, [n], ms, peak, l2_bytes=1 << 40)
    a_c = (m + 1) * 4 + nnz * 8 + m * n * 4
    assert g["per_n"][str(n)]["h"] == 1.0 and g["bytes"] == a_c
    assert abs(g["frac"] - a_c / 1e12 * 1e3 / 1.0) < 1e-15
    # B eight times the L2: h = 1/8 and the bound adds 7/8 of every gather
    b = k * n * 4
    g = bench.gather_aware("none", "other", m, nnz, k, [n], ms, peak, l2_bytes=b // 8)
    assert abs(g["per_n"][str(n)]["h"] - 0.125) < 1e-12
    assert abs(g["bytes"] - (a_c + nnz * n * 4 * 0.875)) < 1e-6


def test_ingest_ncu_csv(tmp_path):
    head = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
           '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'
    lines = ["==PROF== noise line\n", head]
    for i, (rd, wr, ns, hit) in enumerate([(1e8, 2e7, 180000, 66.4), (1e9, 1e8, 320000, 35.9),
                                           (3e9, 2.5e8, 550000, 19.5), (7e9, 5e8, 1150000, 10.1)]):
        kn = f"void spmm::merge_kernel_wide<float, float, float, 4, {2 ** i}>(spmm::MergeArgs)"
        for name, unit, val in (("dram__bytes_read.sum", "byte", f"{rd:,.0f}"), ("dram__bytes_write.sum", "byte", f"{wr:.0f}"),
                                ("gpu__time_duration.sum", "ns", str(ns)), ("lts__t_sector_hit_rate.pct", "%", str(hit))):
            lines.append(f'"{i}","1","python","h","{kn}","1","7","(256, 1, 1)","(912, 1, 1)","0","10.3","Command line profiler metrics","{name}","{unit}","{val}"\n')
    src = tmp_path / "t.csv"
    src.write_text("".join(lines))
    out = tmp_path / "t.json"
    assert bench.ingest_ncu(str(src), str(out)) == 0
    d = json.loads(out.read_text())
    assert d["sources_sha256"] == bench.sources_sha256(d["sources"])
    assert d["per_n"]["8"]["dram_read_bytes"] == 100_000_000 and d["per_n"]["128"]["duration_ns"] == 1_150_000
    assert d["per_n"]["64"]["l2_sector_hit_pct"] == 19.5
    assert "--print-units base" in d["command"]
