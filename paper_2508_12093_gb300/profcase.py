"""Small, self-contained GPU workloads for profiler captures (ncu).

    python -m paper_2508_12093_gb300.profcase hmult      # N=2^16, 3 top-level HMult+KS
    python -m paper_2508_12093_gb300.profcase rotate     # N=2^16, 3 top-level rotations
    python -m paper_2508_12093_gb300.profcase levels     # N=2^16, 2 HMults + 2 rotations at levels 23, 12, 4
    python -m paper_2508_12093_gb300.profcase query      # N=2^16, one kurtosis query
    python -m paper_2508_12093_gb300.profcase batch3     # N=2^16, skew/kurt/CV of three columns, one batch
    python -m paper_2508_12093_gb300.profcase stages [dnum[:shape] ...]  # per-kernel-class times (CUDA events)

Each case sets up keys and one ciphertext, runs a few warm-up iterations, then
the profiled iterations, synchronises and prints "ok".
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


SHAPES = {"e16": (16, False, False, False, False, False), "e8": (8, False, False, False, False, False),
          "e8lazy": (8, True, False, False, False, False), "e8lazyshfl": (8, True, True, False, False, False),
          "e8lazymd8": (8, True, False, True, False, False), "e8cols": (8, True, False, True, True, False),
          "e8inv": (8, True, False, True, False, True), "e8all": (8, True, False, True, True, True)}


def stages(specs=("6",), reps=20):
    """Per-kernel-class GPU time (CUDA events on the library's stream, mean of
    `reps` launches) of HMult and rotation at levels 23, 12 and 4, and the
    whole op's median time, for each spec "dnum" or "dnum:shape" (shape: e16,
    e8, e8lazy, e8lazyshfl, e8lazymd8, e8cols, e8inv, e8all: the inner product's words
    per thread, lazy accumulation, shuffle exchanges, 8-word ModDown CHUNKS pass, COLS
    passes, first inverse passes); one JSON line each."""
    import json
    import torch
    import paper_2508_12093_gb300 as pp
    import workloads
    for spec in specs:
        d, _, shape = str(spec).partition(":")
        d = int(d)
        ctx = pp.Context(workloads.PARAMS[f"n16_d{d}"])
        if shape:
            ctx.set_inner_shape(*SHAPES[shape])
        sk, evk = ctx.keygen(2, rotations=[1])
        a = ctx.encrypt_ints(evk, np.arange(ctx.N, dtype=np.int64) % 1000, 9, 0, 2.0 ** 50)
        for lv in (23, 12, 4):
            al = ctx.drop(a, lv)
            for name, op in (("hmult", lambda: ctx.hmult(evk, al, al)), ("rotate", lambda: ctx.rotate(evk, al, 1))):
                for _ in range(3):
                    op()
                ctx.sync()
                ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                      for _ in range(reps)]
                for e0, e1 in ev:
                    e0.record()
                    op()
                    e1.record()
                torch.cuda.synchronize()
                ts = sorted(e0.elapsed_time(e1) * 1000.0 for e0, e1 in ev)
                ctx.prof_start()
                for _ in range(reps):
                    op()
                ctx.sync()
                ctx.prof_stop()
                cls = {}
                for k in ctx.prof_classes():
                    n, ms = ctx.prof_read(k)
                    if n:
                        cls[k] = round(1000.0 * ms / reps, 2)
                print(json.dumps({"dnum": d, "shape": shape or "e16", "op": name, "level": lv,
                                  "median_us": round(ts[len(ts) // 2], 1),
                                  "per_op_us_by_class": cls}), flush=True)
        ctx.close()


def main(case):
    if case == "stages":
        stages(tuple(sys.argv[2:]) or ("6",))
        return
    import paper_2508_12093_gb300 as pp
    import workloads
    ctx = pp.Context(workloads.PARAMS["n16_d6"])
    if case in ("hmult", "rotate"):
        sk, evk = ctx.keygen(2, rotations=[1])
        a = ctx.encrypt_ints(evk, np.zeros(ctx.N, dtype=np.int64), 9, 0, 2.0 ** 50)
        op = (lambda: ctx.hmult(evk, a, a)) if case == "hmult" else (lambda: ctx.rotate(evk, a, 1))
        for _ in range(2):
            op()
        for _ in range(3):
            op()
    elif case == "levels":
        # each op twice at levels 23, 12 and 4 after one warm-up (for a launch list of
        # per-kernel durations: the small grids of the low levels are latency-bound)
        sk, evk = ctx.keygen(2, rotations=[1])
        a = ctx.encrypt_ints(evk, np.arange(ctx.N, dtype=np.int64) % 1000, 9, 0, 2.0 ** 50)
        for lv in (23, 12, 4):
            al = ctx.drop(a, lv)
            for _ in range(3):
                ctx.hmult(evk, al, al)
            for _ in range(3):
                ctx.rotate(evk, al, 1)
    elif case == "query":
        sk, evk = ctx.keygen(2)
        col = ctx.encrypt_column(evk, workloads.lognormal_column(ctx.S, seed=1), 3)
        ctx.query(evk, "kurt", col, opts=dict(B_x=20.0, cheb_log2deg=7, newton_steps=3))
    elif case == "batch3":
        # three separately encrypted columns: every key switch of the batch runs on
        # three items at one level (the first ones: the rotate-and-sums at level 23)
        sk, evk = ctx.keygen(2)
        x = workloads.lognormal_column(ctx.S, seed=1)
        cols = [ctx.encrypt_column(evk, x, 3 + i) for i in range(3)]
        opts = dict(B_x=20.0, cheb_log2deg=7, newton_steps=3)
        ctx.query_batch(evk, [(s, c, None, opts) for s, c in zip(("skew", "kurt", "cv"), cols)])
    else:
        raise SystemExit(f"unknown case {case}")
    ctx.sync()
    print("ok")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "hmult")
