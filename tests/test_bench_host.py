"""Host-side arithmetic of the benchmark (no GPU): the metric's unit count, the pyramid dims,
the method's own bytes behind roofline.method_basis (against the per-term figures of the
byte budget: 4.87 + 8.36 + 6.37 + 0.66 GB for one finest-level step of 10 x 160x192x160),
the whole-job throughput of replicas, the clock record parsed from nvidia-smi samples, the
staleness guard of the committed DRAM-traffic record and the peak-bandwidth fallback."""
import json
import os
import shutil

import pytest

import bench


@pytest.fixture
def c2():
    saved = (bench.WORKLOAD, bench.PARAMS)
    bench.select_workload("c2")
    yield
    bench.WORKLOAD, bench.PARAMS = saved


def test_units_of_a_c2_registration(c2):
    # 100 steps x 90 ordered pairs x (20*24*20 + 40*48*40 + 80*96*80 + 160*192*160) voxels
    assert bench.level_dims((160, 192, 160), 4) == [(20, 24, 20), (40, 48, 40), (80, 96, 80), (160, 192, 160)]
    assert bench.units_per_registration() == 100 * 90 * (9600 + 76800 + 614400 + 4915200) == 50_544_000_000
    assert bench.level_dims((17, 9, 1), 3) == [(5, 3, 1), (9, 5, 1), (17, 9, 1)]


def test_method_bytes_match_the_byte_budget(c2):
    tot, pair = bench.method_bytes()
    assert tot / 1e9 == pytest.approx(2315, rel=1e-3)  # a whole c2 registration
    assert pair == pytest.approx(11 * 100 * 90 * (9600 + 76800 + 614400 + 4915200), rel=1e-12)
    # one step at the finest level: pair part, squarings, compositions, regulariser + Adam
    bench.WORKLOAD = dict(bench.WORKLOAD, n_levels=1, steps=[1])
    tot1, pair1 = bench.method_bytes()
    assert pair1 / 1e9 == pytest.approx(4.87, abs=0.005)
    assert tot1 / 1e9 == pytest.approx(4.87 + 8.36 + 6.37 + 0.66, abs=0.02)


def test_replica_throughput_is_the_whole_job():
    # two replicas of 1e9 units each, 4 steps, slowest rank 2 s: 4 Gvoxel-iters/s
    assert bench.replica_throughput(1e9, 4, 2000.0, 2) == pytest.approx(4.0)
    assert bench.replica_throughput(1e9, 4, 2000.0, 1) == pytest.approx(2.0)
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5


def test_clock_record_from_samples(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2062, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2055, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 345, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # idle sample
            "garbage line"]
    with open(c.path, "w") as fh:
        fh.write("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc, c.fh = Done(), open(os.devnull, "w")
    rec = c.stop()
    assert rec["sm_max_mhz"] == 2070 and rec["samples"] == 4
    assert rec["sm_mhz"] == 2062  # median of the samples under load (idle ones below half the peak dropped)
    assert rec["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(c.path)


def test_traffic_record_is_dropped_when_its_kernel_changes(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2412_14671_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(bench.ROOT, "profiles", "traffic.txt"), tmp_path / "profiles" / "traffic.txt")
    rec_text = open(tmp_path / "profiles" / "traffic.txt").read()
    fields = dict(line.split(":", 1) for line in rec_text.splitlines() if ":" in line and not line.startswith("#"))
    source, function = fields["source"].strip(), fields["function"].strip()
    text = open(os.path.join(bench.ROOT, "paper_2412_14671_gb300", "csrc", source)).read()
    (src_dir / source).write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = bench.traffic_record()
    assert rec is not None and rec["dram_bytes_per_unit"] > rec["algorithmic_bytes_per_unit"] > 0
    # an edit elsewhere in the file keeps the record; an edit inside the kernel drops it
    (src_dir / source).write_text("// another comment\n" + text)
    assert bench.traffic_record() is not None
    body = bench.kernel_text(str(src_dir / source), function)
    (src_dir / source).write_text(text.replace(body, body.replace("{", "{ /* edited */", 1)))
    assert bench.traffic_record() is None


def test_peak_bandwidth_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    with open(tmp_path / "MEASURED_PEAKS.json", "w") as fh:
        json.dump({"hbm_gbs": 6694.8}, fh)
    assert bench.peaks() == (6694.8, "measured")
