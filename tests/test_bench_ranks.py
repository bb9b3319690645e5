"""The benchmark's multi-rank bookkeeping on CPU (gloo, world size 2):
the step time is the maximum over ranks and the throughput counts the
units of every rank (independent replicas, weak scaling)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    w, r, _ = bench.dist_env()
    assert (w, r) == (world, rank)
    d = bench.dist_init(world, use_cuda=False)
    bench.barrier(d)
    local_ms = [10.0, 25.0][rank]
    ms, = bench.reduce_across([local_ms], "max", d, "cpu")
    units, = bench.reduce_across([3.0 * (1 << 20)], "sum", d, "cpu")
    out.put((rank, ms, units))
    d.destroy_process_group()


def test_two_rank_aggregation_with_gloo():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in res:
        assert ms == 25.0
        assert units == 2 * 3.0 * (1 << 20)


def test_single_rank_is_identity():
    import bench

    assert bench.reduce_across([1.5, 2.0], "max", None, "cpu") == [1.5, 2.0]
    assert bench.dist_init(1, use_cuda=False) is None


def test_algorithmic_bytes_model():
    import bench

    ctr = {"query_slabs": 1000, "insert_slabs": 10, "insert_new_slabs": 2, "delete_slabs": 5, "relax_lists": 3,
           "relax_slabs": 4, "relax_edges": 50, "relax_improved": 7, "wcc_slabs": 9, "wcc_edges": 100}
    assert bench.algorithmic_bytes("query", ctr, 800, 1) == pytest.approx(800 * 40.125 + 128000)
    assert bench.algorithmic_bytes("insert", ctr, 10, 2) == 2 * 10 * 76 + 128 * 12
    assert bench.algorithmic_bytes("sssp_rounds", ctr, 1, 1) == 3 * 16 + 128 * 4 + 16 * 50 + 7 * 20
    assert bench.algorithmic_bytes("wcc_hook_all", ctr, 1, 1) == 128 * 9 + 16 * 100
    assert bench.algorithmic_bytes("unknown", ctr, 1, 1) is None
    # the round kernel also unpacks the tree nodes into dist/parent
    assert bench.algorithmic_bytes("sssp_rounds", dict(ctr, unpacked=1000), 1, 1) == (
        3 * 16 + 128 * 4 + 16 * 50 + 7 * 20 + 1000 * 16)
    dec = {"scan_owners": 40, "scan_slabs": 30, "scan_targets": 20, "scan_improved": 5, "walk_vertices": 64,
           "invalidated": 6, "seed_lists": 2, "seed_slabs": 3, "seed_edges": 11, "seed_improved": 1}
    assert bench.algorithmic_bytes("sssp_relax_into_invalid", dec, 1, 1) == 4 * 40 + 136 * 30 + 16 * 20
    assert bench.algorithmic_bytes("sssp_enqueue_invalid", dec, 1, 1) == 5 * 28
    assert bench.algorithmic_bytes("sssp_invalidate_walk", dec, 1, 1) == 64 * 8 + 6 * 8
    assert bench.algorithmic_bytes("sssp_relax_updated", dec, 1, 1) == 2 * 20 + 128 * 3 + 16 * 11 + 1 * 20


def test_every_traffic_family_has_a_byte_model_or_is_staging():
    import bench

    ctr = {name: 1 for name in ["query_slabs", "insert_slabs", "insert_new_slabs", "delete_slabs", "relax_lists",
                                "relax_slabs", "relax_edges", "relax_improved", "invalidated", "wcc_slabs",
                                "wcc_edges", "seed_lists", "seed_slabs", "seed_edges", "seed_improved",
                                "wcc_upd_slabs", "wcc_upd_edges", "scan_owners", "scan_slabs", "scan_targets",
                                "scan_improved", "walk_vertices", "unpacked"]}
    without_model = {f for f in bench.NCU_TRAFFIC if bench.algorithmic_bytes(f, ctr, 1, 1) is None}
    # staging, the change-log seeds and the commit are not roofline families
    assert without_model <= {"stage_dedup", "sssp_invalidate", "update_slab_pointers"}


def test_traffic_reported_only_for_unchanged_kernel_sources(monkeypatch):
    import bench

    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"sssp_rounds": 123})
    monkeypatch.setattr(bench, "NCU_TRAFFIC_SOURCES_SHA", bench.kernel_sources_sha())
    assert bench.ncu_traffic("sssp_rounds") == 123
    assert bench.ncu_traffic("query") is None
    monkeypatch.setattr(bench, "NCU_TRAFFIC_SOURCES_SHA", "0" * 64)
    assert bench.ncu_traffic("sssp_rounds") is None


def test_bench_arguments_and_workload_names():
    """Every study the benchmark offers is selectable, the road study's
    sizes and Near-Far width are arguments, and the default is the
    power-law step with at least three warm-up steps."""
    import bench

    a = bench.parse_args([])
    assert a.workload == "powerlaw" and a.gpus == 1 and a.warmup >= 3
    for w in ("powerlaw", "growth", "served", "road", "analytics", "buckets", "l2", "set"):
        assert bench.parse_args(["--workload", w]).workload == w
    r = bench.parse_args(["--workload", "road", "--road-size", "1024", "--road-batches", "2",
                          "--road-batch-size", "16384", "--road-delta", "4000"])
    assert (r.road_size, r.road_batches, r.road_batch_size, r.road_delta) == (1024, 2, 16384, 4000)
    assert bench.parse_args(["--workload", "road"]).road_delta is None
    with pytest.raises(SystemExit):
        bench.parse_args(["--workload", "nonsense"])
