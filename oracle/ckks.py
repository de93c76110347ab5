"""Exact RNS-CKKS oracle: parameters, keys, encryption, and evaluator ops.

TEST INFRASTRUCTURE. This module is the oracle the GPU path is checked
against; only tests, the smoke check and the benchmark's CPU baseline import
it. It shares no code with the product library.

The paper (Sec. 3.1) uses CKKS as a black box: Add(C), Add(P), Mul(C),
Mul(P), Rot, levels and the scale Delta. Its experimental parameters
(Sec. 7.1) are N = 2^16, 32768 slots, logPQ about 1443 bits, 128-bit
security. Everything below the Add/Mul/Rot interface is the textbook full-RNS
CKKS with hybrid key switching, in these readings (all exact integers; the
only floating point is the encoder and the FP64 scale bookkeeping):

* ring Z_Q[X]/(X^N + 1), Q = q_0 ... q_L, special primes P = p_0 ... p_{K-1};
  ciphertexts are (c0, c1) with c0 + c1*s = Delta*m + e, held here in the
  coefficient domain, limb-major [l+1][N];
* slots: z_j = m(zeta^(5^j)), zeta = exp(i*pi/N), j < N/2;
* rescale: c_i <- (c_i - [c_l]_centred) * q_l^-1 mod q_i (exact rounding of
  c / q_l, q_l odd so there are no ties);
* hybrid key switching with digits I_j = [j*alpha, (j+1)*alpha) of the full
  chain: ModUp by fast base conversion without correction, inner product with
  the switching key over Q_l u P, ModDown
  y_i = (x_i - conv_P->q_i(x_P)) * P^-1 mod q_i;
* HMult = tensor, key switch of d2, add, rescale; Rot = Galois automorphism
  X -> X^(5^r), then key switch of the rotated c1 with the key of s(X^g);
* Mul(P) by a real constant c: the integer round(c * q_l) (exact product,
  ties away from zero), then rescale, so the scale is kept exactly;
* Add(P) by c: round(c * scale) added to the constant coefficient.
"""
import math
from fractions import Fraction

import numpy as np

from ._clib import lib, ptr64, ptri64, ptr32


class ScaleError(ValueError):
    """Add/Sub of operands whose scales differ by more than 2^-20 (relative)."""


class DepthError(ValueError):
    """An operation needs a level below 0 (the modulus chain is exhausted)."""


def round_half_away(fr):
    """Nearest integer to an exact rational, ties away from zero."""
    fr = Fraction(fr)
    m = math.floor(abs(fr) + Fraction(1, 2))
    return -m if fr < 0 else m


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

def _primes_below(bound, M):
    """Primes q = 1 (mod M), q < bound, in decreasing order."""
    c = (bound // M) * M + 1
    if c >= bound:
        c -= M
    while c > M:
        if lib.or_is_prime(c):
            yield c
        c -= M


def _primes_above(bound, M):
    """Primes q = 1 (mod M), q > bound, in increasing order."""
    c = (bound // M) * M + 1
    if c <= bound:
        c += M
    while True:
        if lib.or_is_prime(c):
            yield c
        c += M


class Params:
    """A parameter set: ring degree, prime chain, digit split and scale.

    Prime chain rule (the paper states only N, Delta and logPQ, Sec. 7.1):
    every prime is 1 mod 2N;  q_0 = the largest prime below 2^q0_bits;  the
    special primes are the next n_p primes below 2^p_bits (skipping q_0);
    q_1 .. q_{n_q-1} are the primes closest to 2^q_bits, taken alternately
    above (odd i) and below (even i) so that rescaling drifts the scale as
    little as possible.
    """

    def __init__(self, log_n, n_q, n_p, dnum, q0_bits, q_bits, p_bits, log_scale,
                 sigma=3.2, gauss_bound=19):
        self.log_n = log_n
        self.N = 1 << log_n
        self.S = self.N // 2
        M = 2 * self.N
        q0 = next(_primes_below(1 << q0_bits, M))
        used = {q0}
        p = []
        for c in _primes_below(1 << p_bits, M):
            if c not in used:
                p.append(c)
                used.add(c)
            if len(p) == n_p:
                break
        up, down = _primes_above(1 << q_bits, M), _primes_below(1 << q_bits, M)
        q = [q0]
        while len(q) < n_q:
            gen = up if len(q) % 2 == 1 else down
            c = next(gen)
            while c in used:
                c = next(gen)
            used.add(c)
            q.append(c)
        self.q = q
        self.p = p
        self.L = n_q - 1
        self.K = n_p
        self.dnum = dnum
        self.alpha = -(-n_q // dnum)
        self.scale = float(2.0 ** log_scale)
        self.sigma = sigma
        self.gauss_bound = gauss_bound
        self.P = math.prod(p)

    def digits(self, level):
        """Digit index sets I_j restricted to limbs 0..level."""
        out = []
        for j in range(self.dnum):
            lo, hi = j * self.alpha, min((j + 1) * self.alpha, level + 1)
            if lo < hi:
                out.append(list(range(lo, hi)))
        return out


def find_psi(q, N):
    """Smallest-generator primitive 2N-th root of unity mod q: psi = g^((q-1)/2N)
    for the least g >= 2 with psi^N = -1 (which forces order exactly 2N)."""
    g = 2
    while True:
        psi = pow(g, (q - 1) // (2 * N), q)
        if pow(psi, N, q) == q - 1:
            return psi
        g += 1


# ---------------------------------------------------------------------------
# containers
# ---------------------------------------------------------------------------

class Ct:
    """Ciphertext (c0, c1) at `level` (limbs 0..level), coefficient domain."""

    def __init__(self, c0, c1, level, scale):
        self.c0, self.c1, self.level, self.scale = c0, c1, level, float(scale)

    def copy(self):
        return Ct(self.c0.copy(), self.c1.copy(), self.level, self.scale)


class SwitchKey:
    """Hybrid switching key: for each digit j, (b_j, a_j) over Q_L u P, in the
    coefficient domain ([L+1+K][N]), plus their transforms for the oracle's
    own products."""

    def __init__(self, b, a, b_ntt, a_ntt):
        self.b, self.a, self.b_ntt, self.a_ntt = b, a, b_ntt, a_ntt


# ---------------------------------------------------------------------------
# the scheme
# ---------------------------------------------------------------------------

PURPOSE_SECRET, PURPOSE_SWK_A, PURPOSE_SWK_E = 1, 2, 3
PURPOSE_ENC_U, PURPOSE_ENC_E0, PURPOSE_ENC_E1 = 4, 5, 6
PURPOSE_PK_A, PURPOSE_PK_E = 7, 8


class Ckks:
    def __init__(self, params):
        self.prm = params
        self.N = params.N
        self.primes = list(params.q) + list(params.p)   # global prime index t
        self.psi = [find_psi(t, self.N) for t in self.primes]
        self.cdt = np.zeros(params.gauss_bound, dtype=np.uint64)
        lib.or_cdt_table(params.sigma, params.gauss_bound, ptr64(self.cdt))

    # -- limb bookkeeping ---------------------------------------------------
    def ext_index(self, level):
        """Global prime indices of Q_level u P."""
        return list(range(level + 1)) + list(range(self.prm.L + 1, self.prm.L + 1 + self.prm.K))

    def _arr(self, idx):
        return np.array([self.primes[t] for t in idx], dtype=np.uint64)

    def _psis(self, idx):
        return np.array([self.psi[t] for t in idx], dtype=np.uint64)

    def ntt(self, a, idx):
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib.or_ntt_fwd_batch(ptr64(a), self.N, len(idx), ptr64(self._arr(idx)), ptr64(self._psis(idx)))
        return a

    def intt(self, a, idx):
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        lib.or_ntt_inv_batch(ptr64(a), self.N, len(idx), ptr64(self._arr(idx)), ptr64(self._psis(idx)))
        return a

    def vmul(self, a, b, idx):
        out = np.empty_like(a)
        lib.or_vec_mul(ptr64(np.ascontiguousarray(a)), ptr64(np.ascontiguousarray(b)), ptr64(out),
                       self.N, len(idx), ptr64(self._arr(idx)))
        return out

    def vmul_scalar(self, a, consts, idx):
        """a[l] * consts[l] mod q_l (consts are non-negative Python ints)."""
        out = np.empty_like(a)
        cs = np.array([c % self.primes[t] for c, t in zip(consts, idx)], dtype=np.uint64)
        lib.or_vec_mul_scalar(ptr64(np.ascontiguousarray(a)), ptr64(cs), ptr64(out), self.N,
                              len(idx), ptr64(self._arr(idx)))
        return out

    def polymul(self, a, b, idx):
        out = np.empty_like(a)
        lib.or_poly_mul(ptr64(np.ascontiguousarray(a)), ptr64(np.ascontiguousarray(b)), ptr64(out),
                        self.N, len(idx), ptr64(self._arr(idx)), ptr64(self._psis(idx)))
        return out

    def vadd(self, a, b, idx):
        qs = self._arr(idx)[:, None]
        return (a + b) % qs

    def vsub(self, a, b, idx):
        qs = self._arr(idx)[:, None]
        return (a + (qs - b)) % qs

    def vneg(self, a, idx):
        qs = self._arr(idx)[:, None]
        return (qs - a) % qs

    def to_rns(self, ints, idx):
        """Signed integer coefficients (int64 array or list of Python ints) -> [len(idx)][N]."""
        out = np.empty((len(idx), self.N), dtype=np.uint64)
        for r, t in enumerate(idx):
            q = self.primes[t]
            if isinstance(ints, np.ndarray) and ints.dtype == np.int64:
                out[r] = (ints % np.int64(q)).astype(np.uint64)
            else:
                out[r] = np.array([int(v) % q for v in ints], dtype=np.uint64)
        return out

    def automorph(self, a, g, idx):
        out = np.empty_like(a)
        lib.or_automorph(ptr64(np.ascontiguousarray(a)), ptr64(out), self.N, len(idx),
                         ptr64(self._arr(idx)), g)
        return out

    def bconv(self, a, src, dst):
        out = np.empty((len(dst), self.N), dtype=np.uint64)
        lib.or_bconv(ptr64(np.ascontiguousarray(a)), ptr64(self._arr(src)), len(src), ptr64(out),
                     ptr64(self._arr(dst)), len(dst), self.N)
        return out

    # -- samplers (ChaCha20 streams, see ckks_oracle.c) ----------------------
    def sample_uniform(self, seed, purpose, index, idx):
        out = np.empty((len(idx), self.N), dtype=np.uint64)
        for r, t in enumerate(idx):
            row = np.empty(self.N, dtype=np.uint64)
            lib.or_sample_uniform(seed, purpose, index, t, self.primes[t], self.N, ptr64(row))
            out[r] = row
        return out

    def sample_ternary(self, seed, purpose, index):
        out = np.empty(self.N, dtype=np.int64)
        lib.or_sample_ternary(seed, purpose, index, self.N, ptri64(out))
        return out

    def sample_gauss(self, seed, purpose, index):
        out = np.empty(self.N, dtype=np.int64)
        lib.or_sample_gauss(seed, purpose, index, self.N, ptr64(self.cdt), self.prm.gauss_bound,
                            ptri64(out))
        return out

    # -- encoding (canonical embedding, slots ordered by powers of 5) --------
    def slot_exponents(self):
        M = 2 * self.N
        e = np.empty(self.prm.S, dtype=np.int64)
        v = 1
        for j in range(self.prm.S):
            e[j] = v
            v = (v * 5) % M
        return e

    def encode_ints(self, z, scale):
        """Real slot values z (len <= N/2, zero padded) -> integer coefficients
        m_i = round(scale * (2/N) * Re sum_j z_j zeta^(-i 5^j)), ties away from 0.
        Computed with a length-N complex FFT (library primitive)."""
        N, S = self.N, self.prm.S
        zz = np.zeros(S, dtype=np.complex128)
        zz[:len(z)] = np.asarray(z, dtype=np.float64)
        e = self.slot_exponents()
        w = np.zeros(N, dtype=np.complex128)
        w[(e - 1) // 2] = zz
        w[(2 * N - e - 1) // 2] = np.conj(zz)
        i = np.arange(N)
        zeta_neg = np.exp(-1j * np.pi * i / N)
        m = (zeta_neg * np.fft.fft(w)).real / N
        x = m * scale
        return [round_half_away(Fraction(float(v))) for v in x]

    def decode_ints(self, ints, scale):
        """Integer coefficients (Python ints, centred) -> N/2 real slot values."""
        N = self.N
        i = np.arange(N)
        mf = np.array([float(Fraction(v) / Fraction(scale)) for v in ints], dtype=np.float64)
        y = N * np.fft.ifft(mf * np.exp(1j * np.pi * i / N))
        e = self.slot_exponents()
        return y[(e - 1) // 2].real

    # -- CRT --------------------------------------------------------------------
    def crt_centred(self, limbs, idx):
        """Residues [len(idx)][N] -> centred Python integers in (-Q/2, Q/2]."""
        qs = [self.primes[t] for t in idx]
        Q = math.prod(qs)
        hats = [Q // q for q in qs]
        coef = [h * pow(h % q, -1, q) for h, q in zip(hats, qs)]
        rows = [limbs[r].tolist() for r in range(len(idx))]
        out = []
        for c in range(self.N):
            v = sum(coef[r] * rows[r][c] for r in range(len(idx))) % Q
            out.append(v - Q if v > Q // 2 else v)
        return out

    # -- keys -------------------------------------------------------------------
    def keygen(self, seed, rotations=()):
        """Secret, public key, relinearisation key and Galois keys for `rotations`."""
        prm = self.prm
        s = self.sample_ternary(seed, PURPOSE_SECRET, 0)
        keys = {"s": s}
        qidx = list(range(prm.L + 1))
        s_q = self.to_rns(s, qidx)
        a = self.sample_uniform(seed, PURPOSE_PK_A, 0, qidx)
        e = self.to_rns(self.sample_gauss(seed, PURPOSE_PK_E, 0), qidx)
        pk0 = self.vadd(self.vneg(self.polymul(a, s_q, qidx), qidx), e, qidx)
        keys["pk"] = (pk0, a)
        full = self.ext_index(prm.L)
        s_full = self.to_rns(s, full)
        s2 = self.polymul(s_full, s_full, full)
        keys["relin"] = self.gen_switch_key(seed, s_full, s2, key_id=0)
        keys["rot"] = {}
        for r in rotations:
            g = self.galois_elt(r)
            sg = self.automorph(s_full, g, full)
            keys["rot"][r % prm.S] = self.gen_switch_key(seed, s_full, sg, key_id=g)
        return keys

    def galois_elt(self, r):
        return pow(5, r % self.prm.S, 2 * self.N)

    def gen_switch_key(self, seed, s_full, s_new, key_id):
        """Key switching from s_new to s:  for digit j and limb t of Q_L u P,
        b_j[t] = -a_j s + e_j + [t in I_j] * (P mod q_t) * s_new[t],  a_j uniform."""
        prm = self.prm
        full = self.ext_index(prm.L)
        Pq = [prm.P % self.primes[t] for t in full]
        bs, as_, bn, an = [], [], [], []
        for j, I in enumerate(prm.digits(prm.L)):
            a = self.sample_uniform(seed, PURPOSE_SWK_A, key_id * 64 + j, full)
            e = self.to_rns(self.sample_gauss(seed, PURPOSE_SWK_E, key_id * 64 + j), full)
            b = self.vadd(self.vneg(self.polymul(a, s_full, full), full), e, full)
            for r, t in enumerate(full):
                if t in I:
                    q = self.primes[t]
                    gad = self.vmul_scalar(s_new[r:r + 1], [Pq[r]], [t])
                    b[r] = (b[r] + gad[0]) % np.uint64(q)
            bs.append(b)
            as_.append(a)
            bn.append(self.ntt(b, full))
            an.append(self.ntt(a, full))
        return SwitchKey(bs, as_, bn, an)

    # -- encryption ---------------------------------------------------------
    def encrypt_ints(self, pk, m_ints, seed, index, scale=None):
        """Public-key encryption of integer coefficients m at the top level:
        (u*pk0 + e0 + m, u*pk1 + e1) with u ternary and e0, e1 Gaussian."""
        prm = self.prm
        qidx = list(range(prm.L + 1))
        u = self.to_rns(self.sample_ternary(seed, PURPOSE_ENC_U, index), qidx)
        e0 = self.to_rns(self.sample_gauss(seed, PURPOSE_ENC_E0, index), qidx)
        e1 = self.to_rns(self.sample_gauss(seed, PURPOSE_ENC_E1, index), qidx)
        m = self.to_rns(m_ints, qidx)
        c0 = self.vadd(self.vadd(self.polymul(u, pk[0], qidx), e0, qidx), m, qidx)
        c1 = self.vadd(self.polymul(u, pk[1], qidx), e1, qidx)
        return Ct(c0, c1, prm.L, prm.scale if scale is None else scale)

    def encrypt_column(self, pk, x, seed):
        """A column of n reals -> ceil(n / S) ciphertexts (last one zero padded);
        ciphertext i uses encryption stream index i."""
        S = self.prm.S
        n = len(x)
        cts = []
        for i in range(max(1, -(-n // S))):
            m = self.encode_ints(x[i * S:(i + 1) * S], self.prm.scale)
            cts.append(self.encrypt_ints(pk, m, seed, i))
        return cts

    def decrypt_ints(self, s, ct):
        idx = list(range(ct.level + 1))
        s_q = self.to_rns(s, idx)
        m = self.vadd(ct.c0, self.polymul(ct.c1, s_q, idx), idx)
        return self.crt_centred(m, idx)

    def decrypt(self, s, ct):
        return self.decode_ints(self.decrypt_ints(s, ct), ct.scale)

    # -- evaluator ------------------------------------------------------------
    def drop(self, ct, level):
        if level > ct.level:
            raise ValueError("cannot raise a level")
        return Ct(ct.c0[:level + 1].copy(), ct.c1[:level + 1].copy(), level, ct.scale)

    def _align(self, a, b):
        lv = min(a.level, b.level)
        return self.drop(a, lv), self.drop(b, lv)

    @staticmethod
    def check_scales(sa, sb):
        if abs(sa / sb - 1.0) >= 2.0 ** -20:
            raise ScaleError(f"scale mismatch {sa} vs {sb}")

    def add(self, a, b):
        a, b = self._align(a, b)
        self.check_scales(a.scale, b.scale)
        idx = list(range(a.level + 1))
        return Ct(self.vadd(a.c0, b.c0, idx), self.vadd(a.c1, b.c1, idx), a.level, a.scale)

    def sub(self, a, b):
        a, b = self._align(a, b)
        self.check_scales(a.scale, b.scale)
        idx = list(range(a.level + 1))
        return Ct(self.vsub(a.c0, b.c0, idx), self.vsub(a.c1, b.c1, idx), a.level, a.scale)

    def add_const(self, ct, c):
        """Add(P) of a real constant: round(c * scale) (FP64 product, then exact
        rounding ties away from zero) added to the constant coefficient of c0."""
        m = round_half_away(Fraction(float(c) * ct.scale))
        out = ct.copy()
        for r in range(ct.level + 1):
            q = self.primes[r]
            out.c0[r, 0] = np.uint64((int(out.c0[r, 0]) + m) % q)
        return out

    def mul_int(self, ct, k):
        """Multiply by a (signed) integer; no level or scale change."""
        idx = list(range(ct.level + 1))
        ks = [k % self.primes[t] for t in idx]
        return Ct(self.vmul_scalar(ct.c0, ks, idx), self.vmul_scalar(ct.c1, ks, idx), ct.level, ct.scale)

    def rescale(self, ct):
        """c_i <- (c_i - [c_l]_centred) * q_l^-1 mod q_i, drop limb l; scale / q_l."""
        lv = ct.level
        if lv == 0:
            raise DepthError("rescale at level 0")
        ql = self.primes[lv]
        out = []
        for c in (ct.c0, ct.c1):
            top = c[lv].astype(np.int64)
            cen = np.where(top > ql // 2, top - np.int64(ql), top)
            rows = []
            for i in range(lv):
                q = self.primes[i]
                cr = (cen % np.int64(q)).astype(np.uint64)
                diff = (c[i] + (np.uint64(q) - cr)) % np.uint64(q)
                rows.append(self.vmul_scalar(diff[None, :], [pow(ql, -1, q)], [i])[0])
            out.append(np.stack(rows))
        return Ct(out[0], out[1], lv - 1, ct.scale / ql)

    def mul_const(self, ct, c, target_scale=None):
        """Mul(P) of a real constant followed by a rescale.

        The integer is round(k * q_l) with k = c * (target / scale) in FP64
        (k = c when no target is given), computed exactly and rounded ties away
        from zero; after the rescale the scale is exactly `target` (or the
        input scale)."""
        lv = ct.level
        if lv == 0:
            raise DepthError("mul_const at level 0")
        ql = self.primes[lv]
        if target_scale is None:
            k, tgt = float(c), ct.scale
        else:
            k, tgt = float(c) * (float(target_scale) / ct.scale), float(target_scale)
        m = round_half_away(Fraction(k) * ql)
        out = self.rescale(self.mul_int(ct, m))
        out.scale = tgt
        return out

    def lin_comb(self, cts, coeffs, target_scale):
        """sum_i c_i ct_i with one rescale: the integers m_i = round(k_i q_l),
        k_i = c_i * (target / scale_i) in FP64 (exact product, ties away from
        zero), multiply ciphertexts that share the level l; the sum is rescaled
        once and its scale is exactly `target`."""
        lv = cts[0].level
        if any(ct.level != lv for ct in cts):
            raise ValueError("lin_comb: operands at different levels")
        if lv == 0:
            raise DepthError("lin_comb at level 0")
        ql = self.primes[lv]
        idx = list(range(lv + 1))
        acc0 = np.zeros((lv + 1, self.N), dtype=np.uint64)
        acc1 = np.zeros_like(acc0)
        for ct, c in zip(cts, coeffs):
            k = float(c) * (float(target_scale) / ct.scale)
            t = self.mul_int(ct, round_half_away(Fraction(k) * ql))
            acc0 = self.vadd(acc0, t.c0, idx)
            acc1 = self.vadd(acc1, t.c1, idx)
        out = self.rescale(Ct(acc0, acc1, lv, target_scale))
        out.scale = float(target_scale)
        return out

    def tensor(self, a, b):
        idx = list(range(a.level + 1))
        d0 = self.polymul(a.c0, b.c0, idx)
        d1 = self.vadd(self.polymul(a.c0, b.c1, idx), self.polymul(a.c1, b.c0, idx), idx)
        d2 = self.polymul(a.c1, b.c1, idx)
        return d0, d1, d2

    def key_switch(self, d, key, level):
        """Hybrid key switching of the polynomial d (coefficient domain, limbs 0..level)."""
        prm = self.prm
        ext = self.ext_index(level)
        # rows of the full-chain key that belong to Q_level u P
        key_rows = list(range(level + 1)) + list(range(prm.L + 1, prm.L + 1 + prm.K))
        acc0 = np.zeros((len(ext), self.N), dtype=np.uint64)
        acc1 = np.zeros((len(ext), self.N), dtype=np.uint64)
        for j, I in enumerate(prm.digits(level)):
            targets = [t for t in ext if t not in I]
            conv = self.bconv(d[I], I, targets)
            dt = np.empty((len(ext), self.N), dtype=np.uint64)
            for r, t in enumerate(ext):
                dt[r] = d[t] if t in I else conv[targets.index(t)]
            dtn = self.ntt(dt, ext)
            acc0 = self.vadd(acc0, self.vmul(dtn, key.b_ntt[j][key_rows], ext), ext)
            acc1 = self.vadd(acc1, self.vmul(dtn, key.a_ntt[j][key_rows], ext), ext)
        u0, u1 = self.intt(acc0, ext), self.intt(acc1, ext)
        return self.mod_down(u0, level), self.mod_down(u1, level)

    def mod_down(self, u, level):
        """y_i = (u_i - conv_{P -> q_i}(u_P)) * P^-1 mod q_i, i <= level."""
        prm = self.prm
        qidx = list(range(level + 1))
        pidx = list(range(prm.L + 1, prm.L + 1 + prm.K))
        conv = self.bconv(u[level + 1:], pidx, qidx)
        diff = self.vsub(u[:level + 1], conv, qidx)
        pinv = [pow(prm.P % self.primes[i], -1, self.primes[i]) for i in qidx]
        return self.vmul_scalar(diff, pinv, qidx)

    def relinearize(self, d0, d1, d2, level, key):
        k0, k1 = self.key_switch(d2, key, level)
        idx = list(range(level + 1))
        return self.vadd(d0, k0, idx), self.vadd(d1, k1, idx)

    def hmult(self, a, b, keys):
        """Mul(C): tensor -> key switch d2 -> add -> rescale; scale (sa*sb)/q_l."""
        a, b = self._align(a, b)
        if a.level == 0:
            raise DepthError("hmult at level 0")
        d0, d1, d2 = self.tensor(a, b)
        c0, c1 = self.relinearize(d0, d1, d2, a.level, keys["relin"])
        ct = Ct(c0, c1, a.level, a.scale * b.scale)
        out = self.rescale(ct)
        out.scale = (a.scale * b.scale) / self.primes[a.level]
        return out

    def rotate(self, ct, r, keys):
        """Rot by r: slot j of the result holds slot j + r of the input."""
        r %= self.prm.S
        if r == 0:
            return ct.copy()
        g = self.galois_elt(r)
        idx = list(range(ct.level + 1))
        c0 = self.automorph(ct.c0, g, idx)
        c1 = self.automorph(ct.c1, g, idx)
        k0, k1 = self.key_switch(c1, keys["rot"][r], ct.level)
        return Ct(self.vadd(c0, k0, idx), k1, ct.level, ct.scale)

    def rotsum(self, ct, keys):
        """Rotate-and-sum over all N/2 slots: log2(N/2) steps ct += Rot(ct, 2^i);
        every slot of the result holds the total."""
        for i in range(self.prm.log_n - 1):
            ct = self.add(ct, self.rotate(ct, 1 << i, keys))
        return ct
