// eval.cu -- evaluator operations on device-resident ciphertexts.
//
// Ciphertexts stay in the evaluation (NTT) domain. Readings of the CKKS ops
// the paper uses as a black box (Sec. 3.1):
//  * HMult = tensor -> hybrid key switch of d2 with the relinearisation key
//    -> add -> rescale; scale (s_a s_b) / q_l;
//  * key switch = iNTT(d) -> ModUp (fast base conversion per digit) -> NTT ->
//    inner product with the key over Q_l u P -> ModDown;
//  * Rot(r) = automorphism X -> X^(5^r) of (c0, c1) then key switch of the
//    rotated c1 with the Galois key;
//  * Mul(P) by a real constant = integer round(k q_l) then rescale (scale kept
//    or steered to a target); Add(P) = round(c * scale) added to every slot.
#include <cmath>

#include "ctx.cuh"

namespace ppst {

static void check_scales(double sa, double sb)
{
    if (!(std::fabs(sa / sb - 1.0) < 0x1p-20))
        throw_err(PPST_E_SCALE, "scale mismatch " + std::to_string(sa) + " vs " + std::to_string(sb));
}

CtObj *ev_add(Ctx &c, const CtObj &a, const CtObj &b, bool sub)
{
    const int lv = std::min(a.level, b.level);
    check_scales(a.scale, b.scale);
    CtObj *o = ct_new(c, lv, a.scale);
    k_add(c, a, b, *o, sub);
    return o;
}

static ConstVec residues(const Ctx &c, __int128 m, int nl)
{
    ConstVec cv;
    for (int i = 0; i < nl; i++) {
        cv.c[i] = h_mod_i128(m, c.primes[i]);
        cv.sh[i] = h_shoup(cv.c[i], c.primes[i]);
    }
    return cv;
}

CtObj *ev_add_const(Ctx &c, const CtObj &a, double x)
{
    const __int128 m = h_round_away(x * a.scale);
    CtObj *o = ct_new(c, a.level, a.scale);
    k_add_scalar_c0(c, a, residues(c, m, a.level + 1), *o);
    return o;
}

CtObj *ev_mul_int(Ctx &c, const CtObj &a, int64_t k)
{
    CtObj *o = ct_new(c, a.level, a.scale);
    k_mul_scalar_ct(c, a, residues(c, (__int128)k, a.level + 1), *o);
    return o;
}

CtObj *ev_rescale(Ctx &c, const CtObj &a)
{
    if (a.level < 1) throw_err(PPST_E_DEPTH, "rescale at level 0");
    ensure_workspace(c);
    CtObj *o = ct_new(c, a.level - 1, a.scale / (double)c.primes[a.level]);
    k_rescale(c, a, *o);
    return o;
}

CtObj *ev_mul_const(Ctx &c, const CtObj &a, double x, double target)
{
    if (a.level < 1) throw_err(PPST_E_DEPTH, "mul_const at level 0");
    ensure_workspace(c);
    const uint64_t ql = c.primes[a.level];
    const double k = target > 0 ? x * (target / a.scale) : x;
    const __int128 m = h_round_mul(k, ql);
    const ConstVec mv = residues(c, m, a.level + 1);
    CtObj *o = ct_new(c, a.level - 1, target > 0 ? target : a.scale);
    try {
        k_rescale_mul(c, a, &mv, *o);
    } catch (...) {
        ct_free(o);
        throw;
    }
    return o;
}

CtObj *ev_lin_comb(Ctx &c, const std::vector<const CtObj *> &cts, const std::vector<double> &coeffs, double target)
{
    if (cts.empty() || cts.size() != coeffs.size() || cts.size() > (size_t)LinArgs::MAXT)
        throw_err(PPST_E_ARG, "lin_comb: 1 to 32 terms");
    const int lv = cts[0]->level;
    for (const CtObj *t : cts)
        if (t->level != lv) throw_err(PPST_E_ARG, "lin_comb: operands at different levels");
    if (lv < 1) throw_err(PPST_E_DEPTH, "lin_comb at level 0");
    if (!(target > 0)) throw_err(PPST_E_ARG, "lin_comb: target scale must be positive");
    ensure_workspace(c);
    const uint64_t ql = c.primes[lv];
    LinArgs args;
    args.n = (int)cts.size();
    for (int k = 0; k < args.n; k++) {
        args.p[k] = cts[k]->d;
        args.m[k] = h_round_mul(coeffs[k] * (target / cts[k]->scale), ql);
    }
    CtObj *t = ct_new(c, lv, target);
    CtObj *o = nullptr;
    try {
        k_lincomb(c, args, lv, *t);
        o = ct_new(c, lv - 1, target);
        k_rescale(c, *t, *o);
    } catch (...) {
        ct_free(t);
        ct_free(o);
        throw;
    }
    ct_free(t);
    return o;
}

CtObj *ev_drop(Ctx &c, const CtObj &a, int level)
{
    (void)c;
    if (level > a.level || level < 0) throw_err(PPST_E_ARG, "drop: bad level");
    return ct_view(a, level);
}

// ev_hmult and ev_rotate (fused key switching) are in ks.cu

CtObj *ev_rotsum(Ctx &c, const EvkObj &k, const CtObj &a)
{
    CtObj *acc = ct_clone(a);
    try {
        for (int i = 0; i < c.logN - 1; i++) {
            CtObj *r = ev_rotate(c, k, *acc, 1 << i);
            CtObj *s = nullptr;
            try {
                s = ev_add(c, *acc, *r, false);
            } catch (...) {
                ct_free(r);
                throw;
            }
            ct_free(r);
            ct_free(acc);
            acc = s;
        }
    } catch (...) {
        ct_free(acc);
        throw;
    }
    return acc;
}

}  // namespace ppst
