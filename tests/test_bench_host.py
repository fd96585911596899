"""Host-side pieces of the benchmark: the kernel-source hash that decides
whether committed ncu traffic figures still describe the kernels, the clock
summary of the timed region, the roofline peak lookup and the whole-job
throughput."""
import bench


def test_code_only_ignores_comments_and_layout():
    a = 'int f(int x) { return x + 1; }  // add one\n'
    b = '/* add one */\nint f(int x)\n{\n    return x + 1;\n}\n'
    assert bench._code_only(a) == bench._code_only(b)


def test_code_only_keeps_code_and_literals():
    base = bench._code_only('int f(int x) { return x + 1; }')
    assert bench._code_only('int f(int x) { return x + 2; }') != base
    # comment markers inside string and character literals are code
    s = bench._code_only('const char *p = "a // b /* c */"; char q = \'/\'; // tail')
    assert s == 'const char *p = "a // b /* c */"; char q = \'/\';'
    e = bench._code_only('const char *p = "say \\"hi\\" // not a comment";')
    assert e == 'const char *p = "say \\"hi\\" // not a comment";'


def test_csrc_hash_is_stable():
    assert bench.csrc_hash() == bench.csrc_hash()
    assert len(bench.csrc_hash()) == 16


def _smi_line(t, sm, mx, reasons=()):
    from datetime import datetime
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    ts = datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join([ts, str(sm), str(mx), "900.0", "0x0"] + flags)


def test_clock_summary_keeps_samples_in_the_timed_window():
    c = bench.ClockSampler(0)
    c.windows = [[1000.0, 1001.0]]
    c.lines = [_smi_line(999.5, 1000, 2070),                        # before the window
               _smi_line(1000.2, 2070, 2070),
               _smi_line(1000.4, 2040, 2070, ("sw_power_cap",)),
               _smi_line(1000.6, 2070, 2070),
               _smi_line(1002.0, 900, 2070, ("hw_slowdown",))]        # after it
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["window"] == "timed region"
    c.windows = [[2000.0, 2001.0]]
    assert c.summary()["reasons"] == ["unsampled"]


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6777.3}')
    assert bench.peaks() == (6777.3, "measured")


def test_traffic_record_only_for_the_kernels_it_was_taken_on(monkeypatch):
    import json
    import os
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    name, ent = next(iter(rec.items()))
    monkeypatch.setattr(bench, "csrc_hash", lambda: ent["csrc_hash"])
    assert bench.traffic_from_profile(name) == ent["dram_bytes_per_launch"]
    assert bench.traffic_from_profile("no such kernel") is None
    monkeypatch.setattr(bench, "csrc_hash", lambda: "0" * 16)
    assert bench.traffic_from_profile(name) is None


def test_job_throughput_counts_every_rank():
    assert bench.job_throughput(2e9, 4, 1.0) == 8.0


def test_sector_floor_matches_a_byte_count_from_the_oracle():
    # faces of a 16^3 float64 grid: the floor from the library's segment
    # lists equals a byte-by-byte count over the oracle's typemaps
    import numpy as np

    import inputs
    import oracle
    import paper_2402_12274_gb300 as dte
    n = 16
    specs = inputs.halo_face_specs(n, 2)
    faces = [dte.Datatype.from_spec(s).commit() for s in specs]
    packed = sum(f.size for f in faces)
    got = bench.sector_floor(faces, n ** 3 * 8, packed)
    cov = np.zeros(n ** 3 * 8, bool)
    for s in specs:
        d, ln = oracle.from_spec(s).iov_elements(1)
        for a, b in zip(d, ln):
            cov[a:a + b] = True
    per_sector = cov.reshape(-1, 32).sum(axis=1)
    touched = int(np.count_nonzero(per_sector))
    partial = int(np.count_nonzero((per_sector > 0) & (per_sector < 32)))
    assert got["touched_sectors"] == touched and got["partial_sectors"] == partial
    assert got["pack"] == 32 * touched + packed
    assert got["unpack"] == packed + 32 * touched + 32 * partial


def test_csrc_hash_covers_every_kernel_source_but_the_request_loop():
    import os
    d = os.path.join(bench.ROOT, "paper_2402_12274_gb300", "csrc")
    assert set(bench.KERNEL_SOURCES) == set(os.listdir(d)) - {"server.cu"}
