"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas, weak scaling).

Each rank of a torchrun launch advances its own cavity; the ranks meet only at a barrier and at
the max-reduction of their timed windows.  These tests run that host logic with the gloo backend
and world size 2, and check the reference arm's rank handling.
"""
import argparse
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        bench.barrier(world)
        # each rank's timed window; the job is as slow as its slowest rank
        t = 0.5 + 0.25 * rank
        t_max = bench.reduce_max(t, world)
        args = argparse.Namespace(steps=1, warmup=0)
        ref = bench.run_reference(args)
        out[rank] = (t_max, bench.job_mlups(1000, 10, world, t_max), ref is None)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slowest_window():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    assert res[0][0] == res[1][0] == 0.75
    # whole-job value: both ranks' node updates over the slowest window
    assert res[0][1] == pytest.approx(1000 * 10 * 2 / 0.75 / 1e6)
    # the reference arm runs on rank 0 only
    assert res[0][2] is False and res[1][2] is True


def test_single_rank_helpers_are_identities():
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench.job_mlups(100, 10, 1, 2.0) == pytest.approx(5e-4)


@pytest.mark.parametrize("argv", [["--batch-launch", "64x1x160"],
                                  ["--only", "batched", "--batch-launch", "64x1"],
                                  ["--warmup", "2"]])
def test_bench_rejects_bad_arguments(argv):
    """A fixed batch launch needs --only batched and three sizes; fewer than 3 warm-up steps is refused."""
    with pytest.raises(SystemExit) as e:
        bench.main(argv)
    assert e.value.code == 2


def test_fp64_roofline_uses_the_counted_operations():
    r = bench.fp64_alu_roofline(500.0, "d3q27")
    assert r["bound"] == "alu"
    assert r["achieved"] == pytest.approx(500.0 * bench.FP64_OPS_PER_NODE["d3q27"] / 1e3, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)


def test_fp64_roofline_takes_the_device_and_the_sampled_clock():
    r = bench.fp64_alu_roofline(500.0, "d2q9", sms=148, clock_ghz=1.9, clock_kind="sampled")
    assert r["peak"] == pytest.approx(148 * bench.FP64_LANE_OPS_PER_SM_CLK * 1.9, rel=1e-3)
    assert "148 SMs" in r["peak_kind"] and "1.900 GHz" in r["peak_kind"]


def test_compact_records_close_the_bench_line():
    """Every form's figures sit at the end of the JSON line, in a short table."""
    line = {"value": 17500.0, "dtype": "f32", "roofline": {"achieved": 5900.0, "frac": 0.87, "bound": "hbm"},
            "config": {"nx": 256, "ny": 256, "nz": 256}}
    forms = [{"lattice": "D3Q27+D3Q15", "precision": "fp64", "box": [256, 256, 256], "mlups": 560.0,
              "gbs": 376.3, "hbm_frac": 0.055, "g_attractors": "option A", "l2_resident": False,
              "roofline": {"frac": 0.87}},
             {"lattice": "D2Q9+D2Q9", "precision": "fp32", "box": [1024, 512, 1], "mlups": 49000.0,
              "gbs": 7056.0, "hbm_frac": 1.04, "g_attractors": "option A", "l2_resident": True}]
    nu = [{"case": "2D cavity 64x64, Ra 1e4, Pr 0.71, 20000 steps",
           "nu_hot_mean": {"fp64": 2.24, "fp32": 2.2401, "fp16s": 2.242},
           "rel_vs_fp64": {"fp32": 7.1e-5, "fp16s": 1.1e-3}}]
    batched = {"nodes": 6303744, "mlups": 43500.0, "gbs": 6264.0, "hbm_frac": 0.92, "speedup_vs_unbatched": 1.6}
    adjoint = {"adjoint_ms_per_step": 0.03, "forward_ms_per_step": 0.003, "adjoint_over_forward": 10.0}
    out = bench.append_secondary(dict(line), forms, nu, batched, adjoint, {"value": 4.2})
    keys = list(out)
    assert keys[-2:] == ["nu_accuracy", "per_form"]
    pf = out["per_form"]
    assert [p["form"] for p in pf] == ["3D f32 (headline)", "3D fp64", "2D fp32",
                                       "2D fp32 batched ensemble", "2D adjoint 256x256 (double-float VJP)"]
    assert pf[1]["alu_frac"] == 0.87 and pf[1]["bound"] == "fp64 alu"
    assert "L2" in pf[2]["note"]
    assert out["nu_accuracy"][0] == {"case": "2D cavity 64x64, Ra 1e4", "nu_fp64": 2.24,
                                     "fp32_rel": 7.1e-5, "fp16s_rel": 1.1e-3}
    assert len(json.dumps({k: out[k] for k in keys[-2:]})) < 2500


def test_reference_arm_reports_the_native_config(capsys):
    """The oracle arm times the same workload: its config is the native arm's, key for key."""
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS"
    assert line["config"] == bench.bench_config(bench.WORKLOAD, 1, 1)
    assert line["config"]["bytes_per_node_update"] == 336.0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
