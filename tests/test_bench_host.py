"""Host-side logic of bench.py without a GPU: the multi-rank reductions
(world size 2 over gloo on CPU), the reference arm's JSON line, the roofline
arithmetic and the freshness rule of the recorded DRAM traffic."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    bench.dist_init("gloo")
    assert bench.world() == (rank, world, rank)
    mx = bench.dist_reduce(10.0 + rank, "max", "cpu")
    sm = bench.dist_reduce(float(rank + 1), "sum", "cpu")
    bench.dist_barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"max": mx, "sum": sm}, fh)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_reductions_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got == {"max": 11.0, "sum": 3.0}


def test_reference_arm_line(monkeypatch, capsys):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.main(["--impl", "reference", "--workload", "single", "--steps", "2", "--warmup", "0"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "pairs/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    args = bench.argparse.Namespace(workload="single", precision=None, protocol="greedy")
    assert line["config"] == bench.bench_config(args, 1)


def test_accuracy_flags_a_planted_error():
    """The bench's accuracy check against oracle costs: exact costs pass, a
    relative error above the tolerance fails (the mistake is planted in the
    GPU side's numbers, on the CPU)."""
    import bench
    from paper_2401_07378_gb300 import workloads as wl
    inp = wl.doc_knn(num_docs=6, seed=2, vocab_size=2000)
    import oracle
    rs = [oracle.solve_pair(inp.pair(k), "l2") for k in range(6)]
    orc = {"costs": {k: r.cost for k, r in enumerate(rs)}, "near_ties": 0}
    good = {k: r.cost for k, r in enumerate(rs)}
    acc = bench.accuracy("docs", inp, good, orc, 1e-3, None)
    assert acc["ok"] and acc["pairs_checked"] == 6 and acc["rel_err_vs_fp32_decision_oracle"] == 0.0
    bad = dict(good)
    bad[4] *= 1 + 2e-3
    acc = bench.accuracy("docs", inp, bad, orc, 1e-3, None)
    assert acc["ok"] is False and acc["rel_err_vs_fp32_decision_oracle"] > 1e-3


def test_reference_arm_non_zero_rank_prints_nothing(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main(["--impl", "reference", "--workload", "single", "--steps", "1", "--warmup", "0"])
    assert capsys.readouterr().out.strip() == ""


def test_roofline_rates_against_hand_worked_figures(monkeypatch):
    """The roofline field on made-up launches, worked by hand.  FP32: 7e9
    pairs at d = 3 over 7 launches in 7 ms is 6e9 pipe ops per 1 ms launch,
    6 T op/s, against 100 SMs x 128 lanes x 2,000 MHz = 25.6 T.  Tensor:
    1e12 pairs at d = 64 over 10 launches in 100 ms is 1,280 TFLOP/s against
    a 2,000 TFLOP/s bf16 peak (twice that for FP8)."""
    import bench
    monkeypatch.setattr(bench, "peaks", lambda: {"sm_max_mhz": 2000.0, "bf16_tflops": 2000.0})
    monkeypatch.setattr(bench, "measured_traffic", lambda: 4.5e5)
    r = bench.roofline(3, "fp32", 0, 7e9, 7, 7.0, 14.0, True, 100)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(25.6) and r["achieved"] == pytest.approx(6.0)
    assert r["frac"] == pytest.approx(6.0 / 25.6) and r["share_of_step"] == pytest.approx(0.5)
    assert r["traffic"] == 4.5e5 and r["kernel"] == "k_nns_lowd (K1)"
    r = bench.roofline(64, "bf16", 8, 1e12, 10, 100.0, 100.0, False, 100)
    assert r["bound"] == "tensor" and r["achieved"] == pytest.approx(1280.0)
    assert r["frac"] == pytest.approx(0.64) and r["traffic"] is None and "top-8" in r["kernel"]
    r = bench.roofline(64, "fp8", 16, 1e12, 10, 100.0, 100.0, False, 100)
    assert r["peak"] == pytest.approx(4000.0) and r["frac"] == pytest.approx(0.32) and "top-16" in r["kernel"]


def test_traffic_only_while_the_k1_source_matches(monkeypatch, tmp_path):
    """The DRAM bytes recorded by an ncu capture are reported only while K1's
    source still hashes to the value stored beside them."""
    import bench
    f = tmp_path / "counters.json"
    f.write_text(json.dumps({"source_sha256": "abc", "dram_bytes_per_launch": 123.0}))
    monkeypatch.setattr(bench, "COUNTERS_FILE", str(f))
    monkeypatch.setattr(bench, "k1_source_hash", lambda: "abc")
    assert bench.measured_traffic() == 123.0
    monkeypatch.setattr(bench, "k1_source_hash", lambda: "abd")
    assert bench.measured_traffic() is None
    monkeypatch.setattr(bench, "COUNTERS_FILE", str(tmp_path / "missing.json"))
    assert bench.measured_traffic() is None
