"""Host-side logic that needs no GPU: the replica aggregation of the
benchmark (world size 2 over gloo), the autotuner's parameter family and its
algorithmic byte counts, and the served-latency percentiles."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.replica_max(1.5 + rank, dist)          # rank 1 is the slowest
        out[rank] = (t, bench.whole_job_rate(30, world, t))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_world2():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.5, 30 * 2 / 2.5)


def test_single_rank_aggregation_is_identity():
    import bench
    assert bench.replica_max(3.25, None) == 3.25
    assert bench.whole_job_rate(12, 1, 2.0) == 6.0


def test_percentiles():
    import bench
    xs = list(range(1, 101))
    assert bench.pct(xs, 50) == 51 and bench.pct(xs, 99) == 99 and bench.pct(xs, 100) == 100
    assert bench.pct([], 50) is None


@pytest.mark.parametrize("dnum,mb", [(3, 176.16), (4, 201.33), (6, 251.66), (12, 402.65)])
def test_autotune_family_and_bytes(dnum, mb):
    """K = n_q / dnum special primes; the key-switch byte counts of the N = 2^16
    chain (two input ciphertexts, the key, the output)."""
    import importlib.util
    import workloads
    # by path: the module needs the built library only to measure, not to plan
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("autotune", os.path.join(root, "paper_2508_12093_gb300", "autotune.py"))
    autotune = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(autotune)
    p = autotune.with_dnum(workloads.PARAMS["n16_d6"], dnum)
    assert p["n_p"] * dnum == 24 and p["log_n"] == 16
    assert abs(autotune.ks_bytes(p) / 1e6 - mb) < 0.01
    with pytest.raises(ValueError):
        autotune.with_dnum(workloads.PARAMS["n16_d6"], 5)


def test_batched_workload_shape():
    """The 64-column batched workload: five statistics per column pair (Z-score,
    CV, skewness and kurtosis of each column, Pearson of the pair), B = 20 for the
    lognormal-shaped columns and 1 for the Bernoulli ones."""
    import bench
    cols = [object() for _ in range(bench.BATCH_COLS)]
    qs = bench.batched_queries(cols)
    assert len(qs) == 4 * 64 + 32
    by = {}
    for q in qs:
        by.setdefault(q[0], []).append(q)
    assert {k: len(v) for k, v in by.items()} == {"zscore": 64, "cv": 64, "skew": 64, "kurt": 64, "pcc": 32}
    for q in qs:
        if q[0] == "pcc":
            i, j = q[4]
            assert j == i + 1 and i % 2 == 0 and q[3]["B_x"] == 20.0 and q[3]["B_y"] == 1.0
        else:
            assert q[3]["B_x"] == (20.0 if q[4][0] % 2 == 0 else 1.0)


def test_autotuner_shapes_and_apply():
    """Every measured kernel shape has its own name, and applying a tuned row sets
    exactly its inner-product shape, tile and block-shape threshold (a stand-in
    context records the calls)."""
    from paper_2508_12093_gb300 import autotune
    names = [autotune.shape_name(s) for s in autotune.INNER]
    assert len(set(names)) == len(names)
    assert all(s["tile"] in autotune.TILES and s["words"] in (8, 16) for s in autotune.INNER)

    class Rec:
        def __init__(self):
            self.calls = []

        def set_inner_shape(self, words, **flags):
            self.calls.append(("shape", words, tuple(sorted(flags.items()))))

        def set_tile(self, t):
            self.calls.append(("tile", t))

        def set_pass_blocks(self, b):
            self.calls.append(("blocks", b))

    r = Rec()
    autotune.apply(r, {"inner": dict(words=8, lazy=True, inverse8=True, tile=4), "pass_min_blocks": 912})
    want_flags = tuple(sorted({f: f in ("lazy", "inverse8") for f in autotune.FLAGS}.items()))
    assert r.calls == [("shape", 8, want_flags), ("tile", 4), ("blocks", 912)]
    r = Rec()
    autotune.apply(r, {"tile": 16})  # a row from before the shape search: the 16-word form
    assert r.calls[0] == ("shape", 16, tuple(sorted({f: False for f in autotune.FLAGS}.items())))
    assert r.calls[1] == ("tile", 16) and len(r.calls) == 2
