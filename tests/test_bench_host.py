"""Host-side logic of bench.py that its JSON line rests on, on CPU:
  * a kernel's DRAM traffic is reported only while the sources it was
    captured from are unchanged (otherwise null),
  * the derived FP32 peak and the algorithmic per-site counts,
  * the labels name the smoother storage and outer arithmetic that ran."""
import json
import os
import shutil

import bench
import synth


def _copy_tree(tmp_path):
    """profiles/traffic.json and every source it hashes, under tmp_path."""
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    os.makedirs(tmp_path / "profiles")
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.json"), tmp_path / "profiles" / "traffic.json")
    for entry in t.values():
        for src in entry["sources"]:
            dst = tmp_path / src
            os.makedirs(dst.parent, exist_ok=True)
            shutil.copy(os.path.join(bench.ROOT, src), dst)
    return t


def test_traffic_is_null_once_a_source_changes(tmp_path, monkeypatch):
    t = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    kernel, entry = next(iter(t.items()))
    # the recorded hash is of the files as they were copied: whatever the
    # working tree holds, a copy whose hash matches returns the stored bytes
    import hashlib
    h = hashlib.sha256()
    for src in entry["sources"]:
        h.update(open(tmp_path / src, "rb").read())
    entry_matches = h.hexdigest()[:16] == entry["source_sha256_16"]
    got = bench.kernel_traffic(kernel)
    assert got == (entry["bytes_per_launch"] if entry_matches else None)
    # make the copy match, then change one source by a byte: null
    entry["source_sha256_16"] = h.hexdigest()[:16]
    json.dump(t, open(tmp_path / "profiles" / "traffic.json", "w"))
    assert bench.kernel_traffic(kernel) == entry["bytes_per_launch"]
    with open(tmp_path / entry["sources"][-1], "ab") as f:
        f.write(b"\n")
    assert bench.kernel_traffic(kernel) is None
    assert bench.kernel_traffic("no such kernel") is None


def test_peak_and_algorithmic_counts():
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2070 MHz
    assert abs(bench.fp32_alu_peak_tflops(2070.0, 152) - 80.54784) < 1e-9
    # one Schwarz sweep at 4 MR steps: 1848 (residual) + 1500 (Schur and
    # reconstruction) + 4 x 1630 (MR steps)
    assert bench.sap_flops_per_site(4) == 9868
    # apply_D bytes per site: 168 reals (two-row links) x 4 B in FP32, x 2 B in 16 bit
    assert bench.DSLASH_REALS_12 * 4 == 672 and bench.DSLASH_REALS_12 * 2 == 336
    assert bench.DSLASH_REALS * 8 == 1536
    # a sweep reads links 72, A 72, A_ee^-1 36, b 24, x 24 and writes x 24
    assert bench.SAP_REALS_PER_SWEEP == 72 + 72 + 36 + 24 + 24 + 24


def test_config_labels_name_what_ran():
    wl = synth.WORKLOADS[bench.WORKLOAD]
    c = bench.config_of(wl, "f16", "df")
    assert c["workload"] == bench.WORKLOAD
    assert c["smoother_storage"] == "f16"
    assert c["outer"].startswith("double-float")
    c = bench.config_of(wl, "f32", "f64_outer")
    assert c["smoother_storage"] == "f32" and "IEEE FP64" in c["outer"]
    assert list(c["dims_TZYX"]) == [64, 32, 32, 32] and list(c["block_TZYX"]) == [4, 4, 4, 4]
    assert bench.config_of(dict(wl), "f32", "df")["workload"] == "custom"
