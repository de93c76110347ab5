/*
 * ckks_oracle.c -- exact CPU primitives of the RNS-CKKS oracle.
 *
 * TEST INFRASTRUCTURE. This file is part of the oracle that the GPU path is
 * checked against. Only tests, the smoke check and the benchmark's CPU
 * baseline may load it; the product library never does, and the two share no
 * code, headers, tables or constant generators.
 *
 * Everything here is the plain definition written out, in the slowest obvious
 * form: every modular product is `(unsigned __int128)a*b % q`, every loop runs
 * over coefficients one by one. Polynomials are arrays of N uint64 residues
 * (one RNS limb); multi-limb functions take a limb-major array [nl][N].
 *
 * The paper (CKKS as a black box, Sec. 3.1; Add/Mul/Rot notation) leaves all
 * RNS internals open. The readings these functions implement are:
 *   - negacyclic ring Z_q[X]/(X^N+1); transform = evaluation at psi^(2k+1),
 *     psi a primitive 2N-th root of unity mod q (natural order);
 *   - fast base conversion without correction (the hybrid key-switching
 *     ModUp/ModDown building block);
 *   - ChaCha20 (RFC 8439 Sec. 2.3) keyed by SplitMix64, with the samplers for
 *     uniform residues, ternary secrets and a CDT discrete Gaussian.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* scalar modular arithmetic                                                 */
/* ------------------------------------------------------------------------ */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a * b) % q);
}

static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q)
{
    u128 s = (u128)a + b;
    return (uint64_t)(s % q);
}

static uint64_t submod(uint64_t a, uint64_t b, uint64_t q)
{
    return a >= b ? (a - b) % q : (uint64_t)(((u128)a + q - (b % q)) % q);
}

uint64_t or_powmod(uint64_t b, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* inverse modulo a prime, by Fermat's little theorem */
uint64_t or_invmod(uint64_t a, uint64_t q)
{
    return or_powmod(a, q - 2, q);
}

/* Deterministic Miller-Rabin for n < 2^64 (the first twelve prime bases are
 * known to suffice below 3.3e24). */
int or_is_prime(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = or_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------------ */
/* negacyclic transform (one limb)                                           */
/* ------------------------------------------------------------------------ */

static void bit_reverse_permute(uint64_t *a, uint32_t N)
{
    for (uint32_t i = 1, j = 0; i < N; i++) {
        uint32_t bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

/* cyclic DFT over Z_q with root w (order N): A_k = sum_i a_i w^(ik), natural order */
static void cyclic_dft(uint64_t *a, uint32_t N, uint64_t q, uint64_t w)
{
    bit_reverse_permute(a, N);
    for (uint32_t len = 2; len <= N; len <<= 1) {
        uint64_t wl = or_powmod(w, N / len, q);
        for (uint32_t i = 0; i < N; i += len) {
            uint64_t wj = 1;
            for (uint32_t j = 0; j < len / 2; j++) {
                uint64_t u = a[i + j];
                uint64_t v = mulmod(a[i + j + len / 2], wj, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                wj = mulmod(wj, wl, q);
            }
        }
    }
}

/* a_hat[k] = sum_i a[i] * psi^((2k+1) i)  mod q,  k = 0..N-1 (natural order) */
void or_ntt_fwd(uint64_t *a, uint32_t N, uint64_t q, uint64_t psi)
{
    uint64_t p = 1;
    for (uint32_t i = 0; i < N; i++) {
        a[i] = mulmod(a[i], p, q);
        p = mulmod(p, psi, q);
    }
    cyclic_dft(a, N, q, mulmod(psi, psi, q));
}

/* inverse of or_ntt_fwd: a[i] = N^-1 psi^-i sum_k a_hat[k] psi^(-2ik) */
void or_ntt_inv(uint64_t *a, uint32_t N, uint64_t q, uint64_t psi)
{
    uint64_t psi_inv = or_invmod(psi, q);
    cyclic_dft(a, N, q, mulmod(psi_inv, psi_inv, q));
    uint64_t ninv = or_invmod(N % q, q);
    uint64_t p = ninv;
    for (uint32_t i = 0; i < N; i++) {
        a[i] = mulmod(a[i], p, q);
        p = mulmod(p, psi_inv, q);
    }
}

/* limb-major batch versions: a is [nl][N], q/psi are [nl] */
void or_ntt_fwd_batch(uint64_t *a, uint32_t N, uint32_t nl, const uint64_t *q, const uint64_t *psi)
{
    for (uint32_t l = 0; l < nl; l++) or_ntt_fwd(a + (size_t)l * N, N, q[l], psi[l]);
}

void or_ntt_inv_batch(uint64_t *a, uint32_t N, uint32_t nl, const uint64_t *q, const uint64_t *psi)
{
    for (uint32_t l = 0; l < nl; l++) or_ntt_inv(a + (size_t)l * N, N, q[l], psi[l]);
}

/* ------------------------------------------------------------------------ */
/* elementwise limb arithmetic                                               */
/* ------------------------------------------------------------------------ */

/* out[l][i] = a[l][i] * b[l][i] mod q[l] */
void or_vec_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t N, uint32_t nl,
                const uint64_t *q)
{
    for (uint32_t l = 0; l < nl; l++)
        for (uint32_t i = 0; i < N; i++) {
            size_t k = (size_t)l * N + i;
            out[k] = mulmod(a[k], b[k], q[l]);
        }
}

/* out[l][i] = a[l][i] * c[l] mod q[l] */
void or_vec_mul_scalar(const uint64_t *a, const uint64_t *c, uint64_t *out, uint32_t N,
                       uint32_t nl, const uint64_t *q)
{
    for (uint32_t l = 0; l < nl; l++)
        for (uint32_t i = 0; i < N; i++) {
            size_t k = (size_t)l * N + i;
            out[k] = mulmod(a[k], c[l] % q[l], q[l]);
        }
}

/* negacyclic product of two RNS polynomials (coefficient domain in and out),
 * through the transform: c = NTT^-1(NTT(a) * NTT(b)) */
void or_poly_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, uint32_t N, uint32_t nl,
                 const uint64_t *q, const uint64_t *psi)
{
    uint64_t *ta = (uint64_t *)malloc(sizeof(uint64_t) * N);
    uint64_t *tb = (uint64_t *)malloc(sizeof(uint64_t) * N);
    for (uint32_t l = 0; l < nl; l++) {
        memcpy(ta, a + (size_t)l * N, sizeof(uint64_t) * N);
        memcpy(tb, b + (size_t)l * N, sizeof(uint64_t) * N);
        or_ntt_fwd(ta, N, q[l], psi[l]);
        or_ntt_fwd(tb, N, q[l], psi[l]);
        for (uint32_t i = 0; i < N; i++) ta[i] = mulmod(ta[i], tb[i], q[l]);
        or_ntt_inv(ta, N, q[l], psi[l]);
        memcpy(out + (size_t)l * N, ta, sizeof(uint64_t) * N);
    }
    free(ta);
    free(tb);
}

/* Galois automorphism X -> X^g (g odd) in the coefficient domain:
 * coefficient i moves to i*g mod 2N, negated when that lands in [N, 2N). */
void or_automorph(const uint64_t *a, uint64_t *out, uint32_t N, uint32_t nl, const uint64_t *q,
                  uint64_t g)
{
    uint64_t twoN = 2ull * N;
    for (uint32_t l = 0; l < nl; l++) {
        const uint64_t *al = a + (size_t)l * N;
        uint64_t *ol = out + (size_t)l * N;
        for (uint32_t i = 0; i < N; i++) {
            uint64_t e = ((u128)i * g) % twoN;
            if (e < N) ol[e] = al[i];
            else ol[e - N] = al[i] == 0 ? 0 : q[l] - al[i];
        }
    }
}

/* Fast base conversion (no correction term):
 *   out[t][c] = sum_i [ in[i][c] * (Qin/qin_i)^-1 ]_{qin_i} * (Qin/qin_i)  mod qout_t
 * where Qin = prod qin. The result is congruent to x + u*Qin for the integer x
 * with residues in[.][c], and 0 <= u < nin. */
void or_bconv(const uint64_t *in, const uint64_t *qin, uint32_t nin, uint64_t *out,
              const uint64_t *qout, uint32_t nout, uint32_t N)
{
    uint64_t *hatinv = (uint64_t *)malloc(sizeof(uint64_t) * nin);
    uint64_t *hat = (uint64_t *)malloc(sizeof(uint64_t) * nin * nout);
    for (uint32_t i = 0; i < nin; i++) {
        uint64_t h = 1;
        for (uint32_t k = 0; k < nin; k++)
            if (k != i) h = mulmod(h, qin[k] % qin[i], qin[i]);
        hatinv[i] = or_invmod(h, qin[i]);
        for (uint32_t t = 0; t < nout; t++) {
            uint64_t ht = 1 % qout[t];
            for (uint32_t k = 0; k < nin; k++)
                if (k != i) ht = mulmod(ht, qin[k] % qout[t], qout[t]);
            hat[(size_t)i * nout + t] = ht;
        }
    }
    for (uint32_t c = 0; c < N; c++) {
        for (uint32_t t = 0; t < nout; t++) {
            uint64_t acc = 0;
            for (uint32_t i = 0; i < nin; i++) {
                uint64_t y = mulmod(in[(size_t)i * N + c], hatinv[i], qin[i]);
                acc = addmod(acc, mulmod(y % qout[t], hat[(size_t)i * nout + t], qout[t]), qout[t]);
            }
            out[(size_t)t * N + c] = acc;
        }
    }
    free(hatinv);
    free(hat);
}

/* ------------------------------------------------------------------------ */
/* pseudo-randomness: SplitMix64 + ChaCha20 block function (RFC 8439 2.3)     */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood 2014; constants of Vigna's splitmix64.c) */
uint64_t or_splitmix64(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* 256-bit ChaCha20 key from a 64-bit seed: four SplitMix64 outputs, each split
 * into two little-endian 32-bit words. */
void or_key_from_seed(uint64_t seed, uint32_t key[8])
{
    uint64_t st = seed;
    for (int i = 0; i < 4; i++) {
        uint64_t z = or_splitmix64(&st);
        key[2 * i] = (uint32_t)z;
        key[2 * i + 1] = (uint32_t)(z >> 32);
    }
}

static uint32_t rotl32(uint32_t v, int c) { return (v << c) | (v >> (32 - c)); }

static void quarter_round(uint32_t *x, int a, int b, int c, int d)
{
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 16);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 12);
    x[a] += x[b]; x[d] ^= x[a]; x[d] = rotl32(x[d], 8);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = rotl32(x[b], 7);
}

/* RFC 8439 Sec. 2.3: constants, key, block counter, nonce -> 20 rounds -> add */
void or_chacha20_block(const uint32_t key[8], uint32_t counter, const uint32_t nonce[3],
                       uint32_t out[16])
{
    uint32_t s[16] = {0x61707865u, 0x3320646eu, 0x79622d32u, 0x6b206574u,
                      key[0], key[1], key[2], key[3], key[4], key[5], key[6], key[7],
                      counter, nonce[0], nonce[1], nonce[2]};
    uint32_t x[16];
    memcpy(x, s, sizeof x);
    for (int r = 0; r < 10; r++) {
        quarter_round(x, 0, 4, 8, 12);
        quarter_round(x, 1, 5, 9, 13);
        quarter_round(x, 2, 6, 10, 14);
        quarter_round(x, 3, 7, 11, 15);
        quarter_round(x, 0, 5, 10, 15);
        quarter_round(x, 1, 6, 11, 12);
        quarter_round(x, 2, 7, 8, 13);
        quarter_round(x, 3, 4, 9, 14);
    }
    for (int i = 0; i < 16; i++) out[i] = x[i] + s[i];
}

/* 64-bit word k (0..7) of block `counter` of the stream (seed, nonce) */
static void block_words(uint64_t seed, uint32_t counter, const uint32_t nonce[3], uint64_t w[8])
{
    uint32_t key[8], o[16];
    or_key_from_seed(seed, key);
    or_chacha20_block(key, counter, nonce, o);
    for (int k = 0; k < 8; k++) w[k] = (uint64_t)o[2 * k] | ((uint64_t)o[2 * k + 1] << 32);
}

/* Uniform residues mod q: coefficient c reads block c/4, words 2r (low) and
 * 2r+1 (high), r = c mod 4, and reduces the 128-bit integer mod q. */
void or_sample_uniform(uint64_t seed, uint32_t purpose, uint32_t index, uint32_t limb,
                       uint64_t q, uint32_t N, uint64_t *out)
{
    uint32_t nonce[3] = {purpose, index, limb};
    uint64_t w[8];
    for (uint32_t c = 0; c < N; c++) {
        if (c % 4 == 0) block_words(seed, c / 4, nonce, w);
        uint32_t r = c % 4;
        u128 v = ((u128)w[2 * r + 1] << 64) | w[2 * r];
        out[c] = (uint64_t)(v % q);
    }
}

/* Ternary coefficients in {-1,0,1}: coefficient c reads word c mod 8 of block
 * c/8 and takes (word mod 3) - 1. */
void or_sample_ternary(uint64_t seed, uint32_t purpose, uint32_t index, uint32_t N, int64_t *out)
{
    uint32_t nonce[3] = {purpose, index, 0};
    uint64_t w[8];
    for (uint32_t c = 0; c < N; c++) {
        if (c % 8 == 0) block_words(seed, c / 8, nonce, w);
        out[c] = (int64_t)(w[c % 8] % 3) - 1;
    }
}

/* Cumulative table of the discrete Gaussian exp(-x^2 / (2 sigma^2)) on
 * [-bound, bound] folded onto |x|: T[k] = floor(2^64 * P(|x| <= k)),
 * k = 0..bound-1. Evaluated in IEEE double in this exact order. */
void or_cdt_table(double sigma, uint32_t bound, uint64_t *T)
{
    double tot = exp(-0.0 / (2.0 * sigma * sigma));
    for (uint32_t x = 1; x <= bound; x++) tot += 2.0 * exp(-(double)(x * x) / (2.0 * sigma * sigma));
    double cum = exp(-0.0 / (2.0 * sigma * sigma));
    for (uint32_t k = 0; k < bound; k++) {
        if (k > 0) cum += 2.0 * exp(-(double)(k * k) / (2.0 * sigma * sigma));
        T[k] = (uint64_t)ldexp(cum / tot, 64);
    }
}

/* Gaussian coefficients: coefficient c reads block c/4, words 2r (magnitude
 * draw) and 2r+1 (sign bit), r = c mod 4; |e| = #{k < bound : draw >= T[k]}. */
void or_sample_gauss(uint64_t seed, uint32_t purpose, uint32_t index, uint32_t N,
                     const uint64_t *T, uint32_t bound, int64_t *out)
{
    uint32_t nonce[3] = {purpose, index, 0};
    uint64_t w[8];
    for (uint32_t c = 0; c < N; c++) {
        if (c % 4 == 0) block_words(seed, c / 4, nonce, w);
        uint32_t r = c % 4;
        uint64_t draw = w[2 * r];
        int64_t mag = 0;
        for (uint32_t k = 0; k < bound; k++)
            if (draw >= T[k]) mag++;
        out[c] = (w[2 * r + 1] & 1) ? -mag : mag;
    }
}
