"""The bench's DRAM-traffic record (CPU only): an ncu CSV of k_spec launches
becomes the machine-readable record the bench reads for `roofline.traffic`,
and a record taken on other kernel sources is ignored."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

CSV = '''"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"
"0","1","python","h","void k_summary_max<0>(SumLaunch)","1","7","(256, 1, 1)","(912, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Mbyte","536.90"
"1","1","python","h","void k_spec<0>(ChainLaunch)","1","7","(128, 1, 1)","(912, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Mbyte","40.00"
"1","1","python","h","void k_spec<0>(ChainLaunch)","1","7","(128, 1, 1)","(912, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","Kbyte","1,000.00"
"1","1","python","h","void k_spec<0>(ChainLaunch)","1","7","(128, 1, 1)","(912, 1, 1)","0","10.3","Command line profiler metrics","gpu__time_duration.sum","us","912.00"
"2","1","python","h","void k_spec<2>(ChainLaunch)","1","7","(128, 1, 1)","(912, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_read.sum","Mbyte","6.00"
"2","1","python","h","void k_spec<2>(ChainLaunch)","1","7","(128, 1, 1)","(912, 1, 1)","0","10.3","Command line profiler metrics","dram__bytes_write.sum","byte","0"
'''


def test_record_from_ncu_csv(tmp_path):
    csv_path = tmp_path / "k.csv"
    csv_path.write_text(CSV)
    out = tmp_path / "rec.json"
    n = 512 << 20
    bench.write_traffic(str(csv_path), n, "ncu ... (test)", out_path=str(out))
    rec = json.loads(out.read_text())
    assert [l["kernel"] for l in rec["launches"]] == ["void k_spec<0>(ChainLaunch)", "void k_spec<2>(ChainLaunch)"]
    assert rec["launches"][0]["dram_bytes"] == 41_000_000  # 40 MB read + 1,000 KB written
    assert rec["launches"][0]["time_ns"] == 912_000.0
    exp = (41e6 / n + 6e6 / n) / 2
    assert abs(rec["dram_bytes_per_input_byte"] - exp) < 1e-12
    # taken on the current sources: the bench uses it
    assert abs(bench.profile_traffic(str(out)) - exp) < 1e-12
    # on other sources: ignored
    rec["source_sha256_16"] = "0" * 16
    out.write_text(json.dumps(rec))
    assert bench.profile_traffic(str(out)) is None
