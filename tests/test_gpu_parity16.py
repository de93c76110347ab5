"""Limb parity against the oracle at N = 2^16, the benchmarked parameter sets.

* every digit count the autotuner chooses from (dnum = 3, 4, 6, 12): HMult and
  a rotation at levels 23, 16, 8 and 1, which covers full and partial last
  digits and each compiled base-conversion width;
* batched launches: three independent HMults and three rotations in one
  key-switch launch sequence, each item against the oracle;
* one whole kurtosis query: tests/test_gpu_stats_query16.py (collected
  later, so its longer oracle job runs while the other tests do).

The oracle side runs in spawned worker processes (tests/oracle_jobs.py),
started when collection selects these tests, and returns per-limb SHA-256
digests of its results; the GPU results are exported and digested the same
way. Bit-exact: every digest must match.
"""
import numpy as np
import pytest

import oracle_jobs as oj
import workloads

pytestmark = pytest.mark.gpu


def check(ctx, g, want, what):
    c0, c1, lv, sc = ctx.ct_export(g)
    got = oj.digest(c0, c1, lv, sc)
    assert (got[0], got[1]) == (want[0], want[1]), (what, got[:2], want[:2])
    bad = [i for i, (a, b) in enumerate(zip(got[2], want[2])) if a != b]
    n = lv + 1
    assert not bad, f"{what}: limbs differ: " + ", ".join(f"c{i // n}[{i % n}]" for i in bad[:12])


def imp(ctx, raw):
    c0, c1, lv, sc = raw
    return ctx.ct_import(c0, c1, lv, sc)


@pytest.mark.oracle16("dnum3", "dnum4", "dnum6", "dnum12")
@pytest.mark.parametrize("dnum", [3, 4, 6, 12])
def test_every_dnum_full_size(dnum):
    import paper_2508_12093_gb300 as pp
    ctx = pp.Context(workloads.PARAMS[f"n16_d{dnum}"])
    sk, evk = ctx.keygen(2, rotations=[oj.ROT])
    want = oj.result(f"dnum{dnum}")
    a, b = imp(ctx, want["a"]), imp(ctx, want["b"])
    for lv in oj.LEVELS:
        al = ctx.drop(a, lv)
        check(ctx, ctx.hmult(evk, al, b), want[("hmult", lv)], f"dnum {dnum} hmult level {lv}")
        check(ctx, ctx.rotate(evk, al, oj.ROT), want[("rot", lv)], f"dnum {dnum} rotation level {lv}")
    # every kernel shape at the top level (words per thread of the inner product, lazy
    # accumulation, shuffle exchanges, 8-word ModDown / COLS / first inverse passes, tile)
    shapes = [dict(words=16, tile=4), dict(words=16, tile=8), dict(words=16, tile=16), dict(words=8, tile=4),
              dict(words=8, tile=8), dict(words=8, lazy=True, tile=4), dict(words=8, lazy=True, tile=8),
              dict(words=8, lazy=True, shuffle=True, tile=4), dict(words=8, shuffle=True, tile=8),
              dict(words=8, lazy=True, moddown8=True, tile=4), dict(words=16, moddown8=True, tile=8),
              dict(words=8, lazy=True, moddown8=True, modup8=True, inverse8=True, tile=4),
              dict(words=16, modup8=True, tile=8), dict(words=16, inverse8=True, tile=8)]
    for sh in shapes:
        sh = dict(sh)
        tile, words = sh.pop("tile"), sh.pop("words")
        ctx.set_inner_shape(words, **sh)
        ctx.set_tile(tile)
        what = f"dnum {dnum}, inner {words} words, {sh}, tile {tile}"
        check(ctx, ctx.hmult(evk, a, b), want[("hmult", 23)], what + ", hmult")
        if words == 8 or sh:
            check(ctx, ctx.rotate(evk, ctx.drop(a, 8), oj.ROT), want[("rot", 8)], what + ", rotation level 8")
            check(ctx, ctx.hmult(evk, ctx.drop(a, 1), b), want[("hmult", 1)], what + ", hmult level 1")
    ctx.set_inner_shape(8, lazy=True, moddown8=True, modup8=True, inverse8=True)  # the defaults
    ctx.set_tile(4)
    # the block shapes the default picks elsewhere: 4 sub-transforms per block at
    # the top level, 16 at level 1
    ctx.set_pass_blocks(1 << 20)
    check(ctx, ctx.hmult(evk, a, b), want[("hmult", 23)], f"dnum {dnum} hmult, 4 per block")
    check(ctx, ctx.rotate(evk, a, oj.ROT), want[("rot", 23)], f"dnum {dnum} rotation, 4 per block")
    ctx.set_pass_blocks(0)
    a1 = ctx.drop(a, 1)
    check(ctx, ctx.hmult(evk, a1, b), want[("hmult", 1)], f"dnum {dnum} hmult level 1, 16 per block")
    check(ctx, ctx.rotate(evk, a1, oj.ROT), want[("rot", 1)], f"dnum {dnum} rotation level 1, 16 per block")
    ctx.set_pass_blocks(228)


@pytest.mark.oracle16("batch")
@pytest.mark.parametrize("lv", [23, 16])
def test_batched_launch_full_size(lv):
    import paper_2508_12093_gb300 as pp
    ctx = pp.Context(workloads.PARAMS["n16_d6"])
    sk, evk = ctx.keygen(2, rotations=[1])
    want = oj.result("batch")
    cts = [imp(ctx, r) for r in want["cts"]]
    xs = [ctx.drop(cts[i], lv) for i in range(3)]
    ys = [cts[(i + 1) % 4] for i in range(3)]
    for i, g in enumerate(ctx.hmult_batch(evk, xs, ys)):
        check(ctx, g, want[("hmult", lv)][i], f"batched hmult item {i} level {lv}")
    for i, g in enumerate(ctx.rotate_batch(evk, xs, 1)):
        check(ctx, g, want[("rot", lv)][i], f"batched rotation item {i} level {lv}")


def test_batch_arguments():
    """Batches of mixed levels or of more than 16 items are refused."""
    import paper_2508_12093_gb300 as pp
    ctx = pp.Context(dict(log_n=12, n_q=6, n_p=2, dnum=3, q0_bits=60, q_bits=40, p_bits=60, log_scale=40))
    sk, evk = ctx.keygen(3, rotations=[1])
    a = ctx.encrypt_column(evk, workloads.uniform_column(100, seed=1), 1).cts()[0]
    with pytest.raises(pp.PpstError) as e:
        ctx.hmult_batch(evk, [a, ctx.drop(a, 3)], [a, a])
    assert e.value.code == -1
    with pytest.raises(pp.PpstError) as e:
        ctx.rotate_batch(evk, [a] * 17, 1)
    assert e.value.code == -1
    g = ctx.hmult_batch(evk, [a, a], [a, a])
    one = ctx.ct_export(ctx.hmult(evk, a, a))
    for x in g:
        y = ctx.ct_export(x)
        assert y[2:] == one[2:] and np.array_equal(y[0], one[0]) and np.array_equal(y[1], one[1])
