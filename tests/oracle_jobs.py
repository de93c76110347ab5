"""Oracle computations at N = 2^16 for the full-size parity tests, run in
spawned worker processes while the rest of the GPU suite runs.

TEST INFRASTRUCTURE: only tests import this module. Each job builds the
oracle's keys from the same seed the GPU side uses, encrypts its inputs, runs
the oracle's ops and returns the inputs (coefficient-domain limbs, for the
GPU to import) and, per expected output, its level, scale and one SHA-256
digest per limb row, so that a mismatch names the limbs that differ without
shipping every expected ciphertext between processes.

The pool is started with the `spawn` method (no fork of a process that may
already hold a CUDA context) by `start()`, which `conftest.py` calls once
collection has selected a test marked `oracle16`.
"""
import hashlib
import multiprocessing as mp
import os
import sys
from concurrent.futures import ProcessPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

LEVELS = (23, 16, 8, 1)
ROT = 5
KURT_OPTS = dict(B=20.0, k=7, t=3)

_pool = None
_futures = {}


def _path():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)


def digest(c0, c1, level, scale):
    """(level, scale, [sha256 of each limb row of c0 then c1])."""
    rows = [hashlib.sha256(r.tobytes()).hexdigest() for r in c0[:level + 1]]
    rows += [hashlib.sha256(r.tobytes()).hexdigest() for r in c1[:level + 1]]
    return level, scale, rows


def _dig(ct):
    return digest(ct.c0, ct.c1, ct.level, ct.scale)


def _raw(ct):
    return ct.c0, ct.c1, ct.level, ct.scale


def job_dnum(dnum):
    """HMult(drop(a, l), b) and Rot(drop(a, l), ROT) at each level of LEVELS,
    key switching with `dnum` digits (partial last digits at levels 16, 8, 1
    for every dnum but 12)."""
    _path()
    import workloads
    from oracle import ckks as ock
    prm = workloads.PARAMS[f"n16_d{dnum}"]
    oc = ock.Ckks(ock.Params(**prm))
    ok = oc.keygen(2, rotations=[ROT])
    a = oc.encrypt_column(ok["pk"], workloads.lognormal_column(32768, seed=1), 3)[0]
    b = oc.encrypt_column(ok["pk"], workloads.uniform_column(32768, seed=2, lo=-1.0, hi=1.0), 4)[0]
    out = {"a": _raw(a), "b": _raw(b)}
    for lv in LEVELS:
        al = oc.drop(a, lv)
        out[("hmult", lv)] = _dig(oc.hmult(al, b, ok))
        out[("rot", lv)] = _dig(oc.rotate(al, ROT, ok))
    return out


def job_batch():
    """Three independent pairs at level 23 and three at level 16 (dnum = 6):
    per item, the oracle's HMult and Rot(., 1)."""
    _path()
    import workloads
    from oracle import ckks as ock
    prm = workloads.PARAMS["n16_d6"]
    oc = ock.Ckks(ock.Params(**prm))
    ok = oc.keygen(2, rotations=[1])
    cts = [oc.encrypt_column(ok["pk"], workloads.lognormal_column(32768, seed=40 + i), 50 + i)[0]
           for i in range(4)]
    out = {"cts": [_raw(c) for c in cts]}
    for lv in (23, 16):
        items = [(oc.drop(cts[i], lv), cts[(i + 1) % 4]) for i in range(3)]
        out[("hmult", lv)] = [_dig(oc.hmult(x, y, ok)) for x, y in items]
        out[("rot", lv)] = [_dig(oc.rotate(x, 1, ok)) for x, _ in items]
    return out


def job_kurt():
    """Kurtosis of a 32,768-row lognormal column at N = 2^16, dnum = 6, with the
    benchmark's settings (B = 20, degree 127, 3 Newton steps): the oracle's
    whole schedule on the encrypted column."""
    _path()
    import workloads
    from oracle import ckks as ock
    from oracle import stats as ost
    prm = workloads.PARAMS["n16_d6"]
    oc = ock.Ckks(ock.Params(**prm))
    ok = oc.keygen(2, rotations=[1 << i for i in range(prm["log_n"] - 1)])
    x = workloads.lognormal_column(32768, seed=1)
    cts = oc.encrypt_column(ok["pk"], x, 3)
    o = KURT_OPTS
    res = ost.kurt(ost.CkksEv(oc, ok), cts, len(x), o["B"], o["k"], o["t"])
    return {"cts": [_raw(c) for c in cts], "n": len(x), "res": _dig(res)}


JOBS = {
    **{f"dnum{d}": (job_dnum, (d,)) for d in (3, 4, 6, 12)},
    "batch": (job_batch, ()),
    "kurt": (job_kurt, ()),
}


def start(names=None):
    """Submit the jobs (all by default) to a spawned process pool."""
    global _pool
    if _pool is not None:
        return
    names = list(JOBS) if names is None else list(names)
    _pool = ProcessPoolExecutor(max_workers=max(1, min(len(names), os.cpu_count() or 1)),
                                mp_context=mp.get_context("spawn"))
    for n in names:
        fn, args = JOBS[n]
        _futures[n] = _pool.submit(fn, *args)


def result(name):
    """The job's return value (submitting it first if it was not started)."""
    if _pool is None:
        start([name])
    if name not in _futures:
        fn, args = JOBS[name]
        _futures[name] = _pool.submit(fn, *args)
    return _futures[name].result()


def shutdown():
    global _pool
    if _pool is not None:
        _pool.shutdown(wait=False, cancel_futures=True)
        _pool = None
