"""Host-side logic of bench.py, on the CPU: the split path's work count, the
hash-gated DRAM traffic, the clock summary and the reference arm's line."""
import json
import types

import pytest

import bench


def _ozaki_work_by_tasks(n, b):
    """The tensor and FP64 flops of the split Cholesky with inverse panels,
    counted task by task: for each k, SYRK(i, k) on the lower 128 x 64 blocks
    of tile (i, i), GEMM_NT_SUB(i, j, k) for k < j < i on all blocks of tile
    (i, j), TRSM_INV(i, k) for i >= k + 2 on all blocks of tile (i, k); a block
    is 36 digit-pair products of 2 * 128 * 64 * b flops.  FP64: POTRF and
    TRTRI b^3 / 3 per k, the critical solve TRSM(k + 1, k) b^3 per k < T - 1."""
    T = -(-n // b)
    rows, cols = -(-b // 128), -(-b // 64)
    lower = sum(1 for r in range(rows) for c in range(cols) if c * 64 < (r + 1) * 128)
    blocks = 0
    for k in range(T):
        for i in range(k + 1, T):
            blocks += lower                       # SYRK(i, k)
            for j in range(k + 1, i):
                blocks += rows * cols             # GEMM_NT_SUB(i, j, k)
            if i >= k + 2:
                blocks += rows * cols             # TRSM_INV(i, k)
    fp64 = sum(b ** 3 / 3 + b ** 3 / 3 + (b ** 3 if k < T - 1 else 0) for k in range(T))
    return blocks * 36 * 2 * 128 * 64 * b, fp64


@pytest.mark.parametrize("n,b", [(512, 128), (1024, 256), (4096, 512), (16384, 512), (2000, 384)])
def test_ozaki_work_counts_every_task(n, b):
    t, f = bench.ozaki_work(n, b)
    t2, f2 = _ozaki_work_by_tasks(n, b)
    assert t == t2
    assert f == pytest.approx(f2, rel=1e-15)


def test_ozaki_work_equals_fp64_flops_times_36_on_full_tiles():
    # On full tiles the split path issues 36 digit-pair products where FP64
    # issues one, so each GEMM_NT_SUB and TRSM_INV tile counts 36 x 2 b^3.
    n, b = 2048, 512
    T = n // b
    gemm_tiles = sum((T - k - 1) * (T - k - 2) // 2 for k in range(T))
    inv_tiles = sum(max(0, T - k - 2) for k in range(T))
    syrk_tiles = T * (T - 1) // 2
    t, _ = bench.ozaki_work(n, b)
    lower = sum(min(2 * (r + 1), b // 64) for r in range(b // 128))
    assert t == 36 * (2 * b ** 3 * (gemm_tiles + inv_tiles) + syrk_tiles * lower * 2 * 128 * 64 * b)


def _profile(tmp_path, h, traffic="123456789"):
    p = tmp_path / "prof.md"
    p.write_text(f"# summary\n\nsource-hash: `{h}`\ntraffic-bytes-per-launch: `{traffic}`\n")
    return str(p)


def test_measured_traffic_only_for_the_captured_sources(tmp_path):
    h = bench.kernel_source_hash()
    assert bench.measured_traffic(_profile(tmp_path, h)) == 123456789
    assert bench.measured_traffic(_profile(tmp_path, "0" * 16)) is None
    assert bench.measured_traffic(str(tmp_path / "missing.md")) is None
    p = tmp_path / "nohash.md"
    p.write_text("traffic-bytes-per-launch: `5`\n")
    assert bench.measured_traffic(str(p)) is None


def test_committed_profiles_carry_a_hash_and_traffic():
    for path in (bench.DRAM_PROFILE, bench.GEMM_DRAM_PROFILE):
        fields = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip().strip("`")
        assert len(fields["source-hash"]) == 16
        assert int(fields["traffic-bytes-per-launch"]) > 0


def test_kernel_source_hash_follows_device_sources_only(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2308_15964_b300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text("kernel 1")
    (csrc / "t.cuh").write_text("tile")
    (csrc / "host.cpp").write_text("host 1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (csrc / "host.cpp").write_text("host 2")       # host-only: same kernels
    assert bench.kernel_source_hash() == h0
    (csrc / "t.cuh").write_text("tile 2")
    h1 = bench.kernel_source_hash()
    assert h1 != h0
    (csrc / "x.h").write_text("header")
    assert bench.kernel_source_hash() != h1


def test_clock_summary(tmp_path):
    c = bench.Clocks(0)
    rows = [
        "0, 2032, 2032, 650.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2017, 2032, 700.25, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2032, 2032, 610.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    c.f.write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0
    assert s["power_w_max"] == 700.25 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c2 = bench.Clocks(0)
    assert c2.summary()["reasons"] == ["no samples"]


def test_reference_arm_line(capsys, monkeypatch):
    monkeypatch.setattr(bench, "REFERENCE_STEP_N", 128)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    args = types.SimpleNamespace(tile=32, warmup=1, steps=2, sigma=1.0, n=16384)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "GFLOP/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["ms_per_step"] == pytest.approx(1e3 * (128 ** 3 / 3) / (line["value"] * 1e9),
                                                rel=1e-9)


def test_reference_arm_other_ranks_print_nothing(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(types.SimpleNamespace(tile=32, warmup=0, steps=1, sigma=1.0, n=128))
    assert capsys.readouterr().out == ""
