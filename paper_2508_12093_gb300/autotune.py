"""Autotuner for the key-switching decomposition (dnum), the inner product's
thread shape and tile, and the transform passes' block shape of a parameter
family.

Hybrid key switching splits the Q chain into dnum digits of alpha = n_q / dnum
primes and extends each digit over K = alpha special primes. Fewer digits
mean fewer ModUp transforms and a smaller evaluation key but a wider base
conversion and a longer ModDown; the key inner product's blocks own 4, 8 or 16
transform chunks (more chunks: longer blocks, fewer per SM) with 16 or 8 words
per thread (8: one warp per chunk, optionally with 128-bit lazy accumulation
of the key products); the other transform passes switch to 8 or 4
sub-transforms per block below a grid-size threshold. Which choice is fastest
is a property of the GPU, so it is measured: for every dnum the tuner builds a
context with its own keys, times top-level HMult + key switch for each inner
shape, then low-level HMults for each block-shape threshold, then a rotation and
one representative statistic query with the best shapes, and picks the dnum
with the fastest query. Results are cached in a JSON file keyed by device and
parameters. Every shape gives bit-identical results (tested).

    python -m paper_2508_12093_gb300.autotune [family] [--cache PATH]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CANDIDATES = (3, 4, 6, 12)
TILES = (4, 8, 16)  # transform chunks per block of the key inner product
# kernel shapes: words per thread of the inner product, 128-bit lazy accumulation,
# warp-shuffle exchanges, 8-word ModDown CHUNKS pass, 8-word COLS passes, 8-word first
# inverse passes, inner-product tile (chunks per block)
FLAGS = ("lazy", "shuffle", "moddown8", "modup8", "inverse8")
INNER = [dict(words=16, tile=4), dict(words=16, tile=8), dict(words=16, tile=16),
         dict(words=8, tile=4), dict(words=8, tile=8), dict(words=8, lazy=True, tile=4),
         dict(words=8, lazy=True, tile=8), dict(words=8, lazy=True, shuffle=True, tile=4),
         dict(words=8, lazy=True, moddown8=True, tile=4), dict(words=8, lazy=True, moddown8=True, tile=8),
         dict(words=8, lazy=True, moddown8=True, modup8=True, tile=4),
         dict(words=8, lazy=True, moddown8=True, inverse8=True, tile=4),
         dict(words=8, lazy=True, moddown8=True, modup8=True, inverse8=True, tile=4)]


def shape_name(sh):
    return f"{sh['words']}" + "".join("+" + f for f in FLAGS if sh.get(f)) + f"/{sh['tile']}"
PASS_BLOCKS = (0, 228, 456, 912)  # grid-size thresholds for smaller transform blocks
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuned.json")


def with_dnum(params, dnum):
    """The same Q chain with dnum digits and K = n_q / dnum special primes."""
    if params["n_q"] % dnum:
        raise ValueError(f"dnum={dnum} does not divide n_q={params['n_q']}")
    return dict(params, dnum=dnum, n_p=params["n_q"] // dnum)


def ks_bytes(params):
    """Algorithmic HBM bytes of one top-level HMult + key switch + rescale: two
    input ciphertexts, the relinearisation key, the output."""
    q, k, d, n = params["n_q"], params["n_p"], params["dnum"], 1 << params["log_n"]
    return (2 * 2 * q + d * 2 * (q + k) + 2 * q) * n * 8


def _timed(op, reps):
    import torch
    for _ in range(3):
        op()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        op()
    e1.record()
    torch.cuda.synchronize()
    return 1000.0 * e0.elapsed_time(e1) / reps  # us


def measure(params, reps=20, query=None, peak_gbs=None):
    """Times one parameter set: top-level HMult + KS, rotation, one query."""
    import paper_2508_12093_gb300 as pp
    import workloads
    ctx = pp.Context(params)
    sk, evk = ctx.keygen(2)  # relinearisation key and the Galois keys of rotations by 2^i
    a = ctx.encrypt_ints(evk, np.zeros(ctx.N, dtype=np.int64), 9, 0, 2.0 ** params["log_scale"])
    out = {"dnum": params["dnum"], "n_p": params["n_p"], "tile_us": {}, "inner_us": {}, "pass_blocks_us": {}}
    shapes = {}
    for sh in INNER:
        if params["log_n"] < 15 and (sh["words"] == 8 or any(sh.get(f) for f in FLAGS)):
            continue  # the 8-word forms exist for 256-point chunks (N = 2^15, 2^16) only
        apply(ctx, {"inner": sh})
        t = _timed(lambda: ctx.hmult(evk, a, a), reps)
        out["inner_us"][shape_name(sh)] = t
        shapes[shape_name(sh)] = sh
        if sh["words"] == 16 and not any(sh.get(f) for f in FLAGS):
            out["tile_us"][str(sh["tile"])] = t
    best = min(out["inner_us"], key=out["inner_us"].get)
    out["inner"] = dict({f: False for f in FLAGS}, **shapes[best])
    out["tile"] = out["inner"]["tile"]
    apply(ctx, out)
    out["hmult_us"] = out["inner_us"][best]  # the best shape's top-level HMult
    low = ctx.drop(a, min(4, params["n_q"] - 1))
    for mb in PASS_BLOCKS:
        ctx.set_pass_blocks(mb)
        out["pass_blocks_us"][str(mb)] = _timed(lambda: ctx.hmult(evk, low, low), reps)
    out["pass_min_blocks"] = int(min(out["pass_blocks_us"], key=out["pass_blocks_us"].get))
    apply(ctx, out)
    out["rotate_us"] = _timed(lambda: ctx.rotate(evk, a, 1), reps)
    out["algorithmic_bytes"] = ks_bytes(params)
    out["hmult_gbs"] = out["algorithmic_bytes"] / (out["hmult_us"] * 1e-6) / 1e9
    if peak_gbs:
        out["hmult_frac_of_hbm"] = out["hmult_gbs"] / peak_gbs
    if query:
        col = ctx.encrypt_column(evk, workloads.lognormal_column(ctx.S, seed=1), 3)
        out["query_us"] = _timed(lambda: ctx.query(evk, query[0], col, opts=query[1]), max(2, reps // 10))
    del a, sk, evk
    ctx.close()
    return out


def apply(ctx, row):
    """Set a measured row's shapes (inner product, transform blocks) on a context."""
    inner = row.get("inner") or {"words": 16, "tile": row.get("tile", 8)}
    ctx.set_inner_shape(inner["words"], **{f: bool(inner.get(f, False)) for f in FLAGS})
    ctx.set_tile(inner["tile"])
    if "pass_min_blocks" in row:
        ctx.set_pass_blocks(row["pass_min_blocks"])


def _key(params):
    import torch
    name = torch.cuda.get_device_name()
    p = {k: params[k] for k in ("log_n", "n_q", "q0_bits", "q_bits", "p_bits", "log_scale")}
    return name + " " + json.dumps(p, sort_keys=True)


QUERY = ("skew", dict(B_x=20.0, cheb_log2deg=7, newton_steps=3))


def tune(params, cache=DEFAULT_CACHE, candidates=CANDIDATES, reps=20, refresh=False, peak_gbs=None, query=QUERY):
    """Returns (best dnum, table of measurements), from the cache when present;
    each table row holds the tile chosen for that dnum."""
    key = _key(params)
    db = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            db = json.load(f)
    if key in db and not refresh:
        return db[key]["dnum"], db[key]["table"]
    table = []
    for d in candidates:
        if params["n_q"] % d:
            continue
        table.append(measure(with_dnum(params, d), reps=reps, peak_gbs=peak_gbs, query=query))
    best = min(table, key=lambda r: (r.get("query_us", r["hmult_us"]), r["hmult_us"]))["dnum"]
    if cache:
        db[key] = {"dnum": best, "table": table, "time": time.strftime("%Y-%m-%d %H:%M:%S")}
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, cache)
    return best, table


def tuned_params(params, cache=DEFAULT_CACHE, **kw):
    """params with the tuned dnum (and its K)."""
    best, _ = tune(params, cache=cache, **kw)
    return with_dnum(params, best)


def tuned_setup(params, cache=DEFAULT_CACHE, **kw):
    """(params with the tuned dnum, its measured row); apply the row's shapes to
    a context of those params with apply(ctx, row)."""
    best, table = tune(params, cache=cache, **kw)
    row = next(r for r in table if r["dnum"] == best)
    return with_dnum(params, best), row


if __name__ == "__main__":
    import argparse
    import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("family", nargs="?", default="n16_d6")
    ap.add_argument("--cache", default=DEFAULT_CACHE)
    ap.add_argument("--refresh", action="store_true")
    a = ap.parse_args()
    best, table = tune(workloads.PARAMS[a.family], cache=a.cache, refresh=a.refresh)
    for r in table:
        print(json.dumps(r))
    print("best dnum:", best)
