/*
 * ci_oracle.c -- plain, single-threaded CPU oracle for the chaotic-iterations
 * (CI) pseudorandom generator of Bahi, Couturier, Guyeux & Heam,
 * "Efficient and Cryptographically Secure Generation of Chaotic Pseudorandom
 * Numbers on GPU" (arXiv 1112.5239).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg load the shared object built from it.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * It is slow on purpose: one lane at a time, one output at a time, in the
 * order the paper's algorithms state, with `unsigned __int128 %` for the BBS
 * modular squaring (the definition, not a fast reduction).
 *
 * What it computes (paper construct -> function):
 *   Eq. (Oplus), x^n = x^{n-1} XOR S^n ............ orc_ci_step
 *   Algorithm 2 (XORshift round) ................... orc_xorshift32_step
 *   xor64, the xor-like of the Sec. 7 experiments ... orc_xor64_step
 *   xor128 with 32-bit words (Sec. 6.2 text) ........ orc_xor128_step
 *   Algorithm 4 (one xor-like per thread, two
 *     combination arrays, mixing with the partners'
 *     previous strategies) ......................... orc_run (xor variant)
 *   BBS x_{n+1} = x_n^2 mod M (Sec. 9.1) ............ orc_bbs_step
 *   Algorithm 5 strategy assembly (w-bit chunks,
 *     two extra shift steps, array_shift) .......... orc_bbs_strategy
 *   Algorithm 5 (16 combination arrays, selection
 *     from the BBS state's low bits) ............... orc_run (BBS variant)
 *   Quarter-circle consumer of output pairs ......... orc_run (counts)
 *   Chaotic Blum-Goldwasser (Sec. 9.2) ............ orc_bg_encrypt, orc_bg_decrypt
 *   Listing 1 (sequential CIPRNG over three 64-bit
 *     xor-likes) and Algorithm 3 (each GPU thread
 *     runs Listing 1, no mixing) ................... orc_listing1_*, orc_naive_*
 *   Algorithm 5 as printed (8 BBS generators per
 *     thread, 16-bit moduli, 4 bits per squaring,
 *     arrays chosen per call, rotation on store) ... orc_run (variant 2)
 *
 * Readings where the paper is silent or garbled (the same readings the CUDA
 * path takes; listed with reasons in the design notes):
 *   - seeding: counter-based splitmix64 replaces the paper's host ISAAC
 *     (Sec. 6.1): draw(seed, i) = mix64(seed + (i + 1) * gamma); lane s owns
 *     indices [s * 2^32, (s + 1) * 2^32).
 *   - synchronous mixing: iteration i reads the partners' strategies of
 *     iteration i - 1 (what warp lockstep gives Algorithm 4's unsynchronised
 *     shared-memory read/write); partner = group * C + comb[offset].
 *   - stream-major output out[s * L + i] = x after the (i + 1)-th update.
 *   - xor64 feeds Algorithm 4 with the low 32 bits of each step (the way
 *     Listing 1 takes "(unsigned int)t" from its 64-bit generators).
 *   - BBS: one generator per lane, w = floor(log2(floor(log2 M))) bits per
 *     squaring, ceil(32 / w) chunks, then Algorithm 5's two shift steps;
 *     combination arrays chosen once from the seed's low bits.
 *   - Algorithm 5 as printed (variant 2): eight generators per lane, each with
 *     its own M = p q of Blum primes from [128, 256) (so x^2 < 2^32); 4 bits per
 *     squaring as printed; per output BBS1..BBS8, then BBS3/BBS1 and BBS7/BBS2
 *     for the two shift steps; the two arrays chosen when a call starts from
 *     generators 1 and 2 (state & 7); at the end of a call generator k moves
 *     to place k + 1 (state and modulus together).
 *
 * Parity pins (the tests that tie this file to the paper and to mathematics):
 *   Table 1 worked example; brute force of the single-cell and subset CI
 *   definitions on tiny widths; exhaustive period 2^32 - 1 of Algorithm 2;
 *   full period of xor128 as a GF(2)-linear map; mixing special cases and a
 *   hand-worked small case; GF(2) linearity; BBS squaring on tiny Blum moduli;
 *   Algorithm 5's 4-bit packing on hand-fed BBS values; quarter-circle counts
 *   against the real-number test; the first outputs of the published
 *   splitmix64, xor128 and xor64 programs from their printed start states; the
 *   output functions of Listing 1's five-word xorshift and xorwow by the
 *   linearity of the word sequences they must give back.  Parity unpinned
 *   (readings, not values fixed by the paper): the counter layout of the
 *   seeding draws, and Listing 1's use of its xor-likes on 64-bit words.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Seeding: splitmix64 (Steele, Lea & Flood, OOPSLA 2014), counter-based.     */
/* ------------------------------------------------------------------------- */

#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

static uint64_t orc_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* The (index + 1)-th output of a splitmix64 generator started at `seed`. */
uint64_t orc_draw(uint64_t seed, uint64_t index)
{
    return orc_mix64(seed + (index + 1) * ORC_GAMMA);
}

/* Draw k of lane s: index s * 2^32 + k. */
static uint64_t orc_lane_draw(uint64_t seed, uint64_t lane, uint64_t k)
{
    return orc_draw(seed, (lane << 32) + k);
}

/* ------------------------------------------------------------------------- */
/* Eq. (Oplus): bit k of the state flips iff bit k of the strategy is 1.      */
/* ------------------------------------------------------------------------- */

uint32_t orc_ci_step(uint32_t x, uint32_t strategy)
{
    return x ^ strategy;
}

/* ------------------------------------------------------------------------- */
/* Strategy sources.                                                          */
/* ------------------------------------------------------------------------- */

/* Algorithm 2: one round of the 32-bit XORshift; returns the new z. */
uint32_t orc_xorshift32_step(uint32_t z)
{
    z = z ^ (z << 13);
    z = z ^ (z >> 17);
    z = z ^ (z << 5);
    return z;
}

/* Exhaustive period from a nonzero start: number of rounds until the orbit
 * returns to its start (stops after `limit` rounds and returns 0). */
uint64_t orc_xorshift32_period(uint32_t start, uint64_t limit)
{
    uint32_t z = start;
    uint64_t n = 0;
    do {
        z = orc_xorshift32_step(z);
        ++n;
        if (n > limit)
            return 0;
    } while (z != start);
    return n;
}

/* xor128 with 32-bit words (the Alg. 4 xor-like per Sec. 6.2): s = {a,b,c,d};
 * the new word d is the output. */
uint32_t orc_xor128_step(uint32_t *s)
{
    uint32_t a = s[0];
    uint32_t tmp = a ^ (a << 11);
    s[0] = s[1];
    s[1] = s[2];
    s[2] = s[3];
    s[3] = s[3] ^ (s[3] >> 19) ^ (tmp ^ (tmp >> 8));
    return s[3];
}

/* xor64 (Marsaglia's 64-bit xorshift, the generator of the Sec. 7
 * measurements): x ^= x << 13; x ^= x >> 7; x ^= x << 17.  Returns the new
 * state; the strategy word is its low 32 bits. */
uint64_t orc_xor64_step(uint64_t x)
{
    x = x ^ (x << 13);
    x = x ^ (x >> 7);
    x = x ^ (x << 17);
    return x;
}

/* BBS (Sec. 9.1): x_{n+1} = x_n^2 mod M, by the definition. */
uint64_t orc_bbs_step(uint64_t y, uint64_t M)
{
    unsigned __int128 sq = (unsigned __int128)y * (unsigned __int128)y;
    return (uint64_t)(sq % (unsigned __int128)M);
}

/* Number of secure low bits per BBS output: floor(log2(floor(log2 M))). */
uint32_t orc_bbs_w(uint64_t M)
{
    uint32_t lg = 0, w = 0;
    while ((M >> lg) > 1)
        ++lg;               /* lg = floor(log2 M) */
    while ((lg >> w) > 1)
        ++w;                /* w = floor(log2 lg) */
    return w;
}

/* ------------------------------------------------------------------------- */
/* Primes for BBS: trial division (the definition of primality).             */
/* ------------------------------------------------------------------------- */

int orc_is_prime(uint64_t n)
{
    if (n < 2)
        return 0;
    if (n % 2 == 0)
        return n == 2;
    for (uint64_t d = 3; d * d <= n; d += 2)
        if (n % d == 0)
            return 0;
    return 1;
}

static uint64_t orc_gcd(uint64_t a, uint64_t b)
{
    while (b) {
        uint64_t r = a % b;
        a = b;
        b = r;
    }
    return a;
}

/* ------------------------------------------------------------------------- */
/* Per-lane state.                                                            */
/* ------------------------------------------------------------------------- */

enum { ORC_VAR_XOR = 0, ORC_VAR_BBS = 1, ORC_VAR_BBS16 = 2 };
enum { ORC_XL_XOR128 = 0, ORC_XL_XORSHIFT32 = 1, ORC_XL_XOR64 = 2 };

typedef struct {
    uint32_t w[4];   /* xor-like words: xor128 {a,b,c,d}; xorshift32 uses w[0];
                        xor64 keeps its state as w[0] (low) and w[1] (high) */
    uint32_t x;      /* CI state x */
    uint32_t tprev;  /* the lane's last strategy (its shared-memory slot)     */
    uint32_t p, q;   /* BBS Blum primes                                      */
    uint64_t M;      /* BBS modulus p*q                                      */
    uint64_t y;      /* BBS state, canonical residue in [0, M)               */
    uint32_t sel1;   /* BBS: first combination array index, in [0, 8)      */
    uint32_t sel2;   /* BBS: second combination array index is 8 + sel2    */
    uint32_t y16[8]; /* variant 2: states of BBS1..BBS8                    */
    uint32_t m16[8]; /* variant 2: their moduli                            */
} orc_lane;

uint32_t orc_lane_size(void) { return (uint32_t)sizeof(orc_lane); }

/* xor variant seeding: draws 0 and 1 fill the xor-like words, draw 2 gives x
 * and the initial shared-memory slot (Alg. 4 loads both with the state). */
static void orc_init_xor_lane(int xl, uint64_t seed, uint64_t lane, orc_lane *L)
{
    memset(L, 0, sizeof *L);
    uint64_t d0 = orc_lane_draw(seed, lane, 0);
    uint64_t d1 = orc_lane_draw(seed, lane, 1);
    uint64_t d2 = orc_lane_draw(seed, lane, 2);
    if (xl == ORC_XL_XOR128) {
        L->w[0] = (uint32_t)d0;
        L->w[1] = (uint32_t)(d0 >> 32);
        L->w[2] = (uint32_t)d1;
        L->w[3] = (uint32_t)(d1 >> 32);
        if ((L->w[0] | L->w[1] | L->w[2] | L->w[3]) == 0)
            L->w[0] = 1;
    } else if (xl == ORC_XL_XOR64) {
        L->w[0] = (uint32_t)d0;
        L->w[1] = (uint32_t)(d0 >> 32);
        if ((L->w[0] | L->w[1]) == 0)
            L->w[0] = 1;
    } else {
        L->w[0] = (uint32_t)d0;
        if (L->w[0] == 0)
            L->w[0] = 1;
    }
    L->x = (uint32_t)d2;
    L->tprev = (uint32_t)(d2 >> 32);
}

/* BBS seeding by rejection: candidate c = 2^30 + (draw >> 34), c |= 3, kept if
 * prime; q likewise and distinct from p; seed v = 2 + draw mod (M - 2) kept if
 * coprime to M; then one draw for x and the initial slot.  The combination
 * arrays are chosen by v's low bits (sel1 = v & 7, sel2 = (v >> 3) & 7). */
static void orc_init_bbs_lane(uint64_t seed, uint64_t lane, orc_lane *L)
{
    memset(L, 0, sizeof *L);
    uint64_t k = 0, d, v;
    uint32_t p, q;
    do {
        d = orc_lane_draw(seed, lane, k++);
        p = (uint32_t)((1ULL << 30) + (d >> 34)) | 3u;
    } while (!orc_is_prime(p));
    do {
        d = orc_lane_draw(seed, lane, k++);
        q = (uint32_t)((1ULL << 30) + (d >> 34)) | 3u;
    } while (!orc_is_prime(q) || q == p);
    uint64_t M = (uint64_t)p * (uint64_t)q;
    do {
        d = orc_lane_draw(seed, lane, k++);
        v = 2 + d % (M - 2);
    } while (orc_gcd(v, M) != 1);
    d = orc_lane_draw(seed, lane, k++);
    L->p = p;
    L->q = q;
    L->M = M;
    L->y = v;
    L->x = (uint32_t)d;
    L->tprev = (uint32_t)(d >> 32);
    L->sel1 = (uint32_t)(v & 7);
    L->sel2 = (uint32_t)((v >> 3) & 7);
}

/* Variant 2 seeding: for each of the eight generators, in order, Blum primes
 * p != q from candidates (128 + draw mod 128) | 3, kept if prime; a seed
 * v = 2 + draw mod (M - 2) coprime to M; then one draw for x and the slot. */
static void orc_init_bbs16_lane(uint64_t seed, uint64_t lane, orc_lane *L)
{
    memset(L, 0, sizeof *L);
    uint64_t k = 0, d, v;
    for (int g = 0; g < 8; ++g) {
        uint32_t p, q;
        do {
            d = orc_lane_draw(seed, lane, k++);
            p = (uint32_t)(128 + d % 128) | 3u;
        } while (!orc_is_prime(p));
        do {
            d = orc_lane_draw(seed, lane, k++);
            q = (uint32_t)(128 + d % 128) | 3u;
        } while (!orc_is_prime(q) || q == p);
        uint64_t M = (uint64_t)p * q;
        do {
            d = orc_lane_draw(seed, lane, k++);
            v = 2 + d % (M - 2);
        } while (orc_gcd(v, M) != 1);
        L->y16[g] = (uint32_t)v;
        L->m16[g] = (uint32_t)M;
    }
    d = orc_lane_draw(seed, lane, k++);
    L->x = (uint32_t)d;
    L->tprev = (uint32_t)(d >> 32);
}

/* Seed lanes [lane0, lane0 + nl) by their global index. */
void orc_init_lanes(int variant, int xl, uint64_t seed, uint64_t lane0, uint64_t nl,
                    orc_lane *lanes)
{
    for (uint64_t i = 0; i < nl; ++i) {
        if (variant == ORC_VAR_BBS)
            orc_init_bbs_lane(seed, lane0 + i, &lanes[i]);
        else if (variant == ORC_VAR_BBS16)
            orc_init_bbs16_lane(seed, lane0 + i, &lanes[i]);
        else
            orc_init_xor_lane(xl, seed, lane0 + i, &lanes[i]);
    }
}

/* ------------------------------------------------------------------------- */
/* Combination arrays (Alg. 4: two; Alg. 5: sixteen), each a permutation of  */
/* [0, C) drawn by Fisher-Yates from splitmix64(comb_seed).                   */
/* ------------------------------------------------------------------------- */

static void orc_permutation(uint32_t C, uint64_t comb_seed, uint64_t *ctr, uint8_t *a)
{
    for (uint32_t i = 0; i < C; ++i)
        a[i] = (uint8_t)i;
    for (uint32_t i = C - 1; i >= 1; --i) {
        uint64_t r = orc_draw(comb_seed, (*ctr)++);
        uint32_t j = (uint32_t)(r % (uint64_t)(i + 1));
        uint8_t tmp = a[i];
        a[i] = a[j];
        a[j] = tmp;
    }
}

/* Writes 2*C bytes (xor) or 16*C bytes (BBS).  For the xor variant the second
 * array is redrawn until comb1[j] != comb2[j] for every j (equal partners would
 * cancel in the XOR); C == 1 has no such pair and keeps the single draw. */
int orc_comb_arrays(int variant, uint32_t C, uint64_t comb_seed, uint8_t *out)
{
    if (C < 1 || C > 32 || (C & (C - 1)))
        return -1;
    uint64_t ctr = 0;
    if (variant == ORC_VAR_BBS || variant == ORC_VAR_BBS16) {
        for (int a = 0; a < 16; ++a)
            orc_permutation(C, comb_seed, &ctr, out + (size_t)a * C);
        return 0;
    }
    orc_permutation(C, comb_seed, &ctr, out);
    for (;;) {
        orc_permutation(C, comb_seed, &ctr, out + C);
        if (C == 1)
            break;
        int clash = 0;
        for (uint32_t j = 0; j < C; ++j)
            if (out[j] == out[C + j])
                clash = 1;
        if (!clash)
            break;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 5 strategy assembly.                                            */
/* ------------------------------------------------------------------------- */

/* Source of BBS outputs: either the lane's generator, or (for the hand-fed
 * pin) a caller-given list of values. */
typedef struct {
    orc_lane *lane;
    const uint64_t *feed;
    uint32_t fed;
} orc_bbs_src;

static uint64_t orc_bbs_next(orc_bbs_src *s)
{
    if (s->feed)
        return s->feed[s->fed++];
    s->lane->y = orc_bbs_step(s->lane->y, s->lane->M);
    return s->lane->y;
}

static uint32_t orc_bbs_strategy_src(orc_bbs_src *s, uint32_t w)
{
    static const uint32_t array_shift[4] = {0u, 1u, 3u, 7u};
    uint32_t mask = (1u << w) - 1u;
    uint32_t chunks = (32u + w - 1u) / w;
    uint32_t t = 0;
    /* fill t w bits at a time ("t <<= 4; t |= BBSk(bbsk) & 15" for w = 4) */
    for (uint32_t c = 0; c < chunks; ++c) {
        t <<= w;
        t |= (uint32_t)(orc_bbs_next(s) & mask);
    }
    /* the two extra shifts: shift by the draw's last 2 bits, then put exactly
     * that many low bits of the next draw in the vacated positions */
    for (int r = 0; r < 2; ++r) {
        uint32_t shift = (uint32_t)(orc_bbs_next(s) & 3u);
        t <<= shift;
        t |= (uint32_t)(orc_bbs_next(s) & array_shift[shift]);
    }
    return t;
}

/* Algorithm 5 as printed: BBSk advances generator k (x <- x^2 mod M_k) and
 * returns it.  Eight 4-bit chunks from BBS1..BBS8, then
 * shift = BBS3 & 3; t <<= shift; t |= BBS1 & array_shift[shift];
 * shift = BBS7 & 3; t <<= shift; t |= BBS2 & array_shift[shift]. */
static uint32_t orc_bbs16_next(orc_lane *L, int k)
{
    L->y16[k] = (uint32_t)(((uint64_t)L->y16[k] * L->y16[k]) % L->m16[k]);
    return L->y16[k];
}

uint32_t orc_bbs16_strategy(orc_lane *L)
{
    static const uint32_t array_shift[4] = {0u, 1u, 3u, 7u};
    uint32_t t = 0, shift;
    for (int k = 0; k < 8; ++k) {
        t <<= 4;
        t |= orc_bbs16_next(L, k) & 15u;
    }
    shift = orc_bbs16_next(L, 2) & 3u;
    t <<= shift;
    t |= orc_bbs16_next(L, 0) & array_shift[shift];
    shift = orc_bbs16_next(L, 6) & 3u;
    t <<= shift;
    t |= orc_bbs16_next(L, 1) & array_shift[shift];
    return t;
}

/* End of a variant-2 call: generator k's state and modulus move to place
 * k + 1, generator 8's to place 1. */
static void orc_bbs16_rotate(orc_lane *L)
{
    uint32_t y = L->y16[7], m = L->m16[7];
    for (int k = 7; k > 0; --k) {
        L->y16[k] = L->y16[k - 1];
        L->m16[k] = L->m16[k - 1];
    }
    L->y16[0] = y;
    L->m16[0] = m;
}

/* Hand-fed form: assembles one strategy word from `feed` (needs
 * ceil(32/w) + 4 values) and reports how many values it used. */
uint32_t orc_bbs_strategy_fed(uint32_t w, const uint64_t *feed, uint32_t *used)
{
    orc_bbs_src s = {NULL, feed, 0};
    uint32_t t = orc_bbs_strategy_src(&s, w);
    if (used)
        *used = s.fed;
    return t;
}

/* ------------------------------------------------------------------------- */
/* Algorithms 4 and 5: mixing and the CI update, synchronous over lanes.      */
/* ------------------------------------------------------------------------- */

/* One synchronous iteration over lanes [0, nl) given this iteration's own
 * strategy words xl[]: every lane reads its two partners' previous strategies,
 * then all slots and states are updated together.  part1/part2 give each
 * lane's partners as lane indices within [0, nl). */
static void orc_mix_ci_iteration(uint64_t nl, const uint32_t *xl, const uint64_t *part1,
                                 const uint64_t *part2, uint32_t *tprev, uint32_t *x,
                                 uint32_t *tnew)
{
    for (uint64_t l = 0; l < nl; ++l)
        tnew[l] = xl[l] ^ tprev[part1[l]] ^ tprev[part2[l]];
    for (uint64_t l = 0; l < nl; ++l) {
        tprev[l] = tnew[l];
        x[l] = orc_ci_step(x[l], tnew[l]);
    }
}

/* Hand-fed mixing: given per-iteration strategy words xl[i * nl + l] and the
 * partner lists, runs L iterations from (x, tprev), writing out[l * L + i]. */
void orc_mix_ci_fed(uint64_t nl, uint64_t L, const uint32_t *xl, const uint64_t *part1,
                    const uint64_t *part2, uint32_t *x, uint32_t *tprev, uint32_t *out)
{
    uint32_t *tnew = (uint32_t *)malloc(sizeof(uint32_t) * (nl ? nl : 1));
    for (uint64_t i = 0; i < L; ++i) {
        orc_mix_ci_iteration(nl, xl + i * nl, part1, part2, tprev, x, tnew);
        for (uint64_t l = 0; l < nl; ++l)
            out[l * L + i] = x[l];
    }
    free(tnew);
}

/* Runs L iterations of the generator on lanes[0..nl) (nl a multiple of C;
 * lanes[0] must be the first lane of a group).  comb holds the combination
 * arrays (2*C bytes for xor, 16*C for BBS).  Writes out[l * L + i] when `out`
 * is not NULL; when `counts` is not NULL adds, per lane, the number of output
 * pairs (out[2k], out[2k+1]) whose 24-bit fixed-point coordinates
 * (a, b) = (o0 >> 8, o1 >> 8) fall inside the quarter circle
 * a^2 + b^2 < 2^48 (L must then be even).  Returns 0, or -1 on bad arguments. */
int orc_run(int variant, int xl, uint32_t C, const uint8_t *comb, orc_lane *lanes,
            uint64_t nl, uint64_t L, uint32_t *out, uint64_t *counts)
{
    if (C < 1 || C > 32 || (C & (C - 1)) || nl % C != 0)
        return -1;
    if (counts && (L & 1))
        return -1;
    uint64_t *p1 = (uint64_t *)malloc(sizeof(uint64_t) * (nl ? nl : 1));
    uint64_t *p2 = (uint64_t *)malloc(sizeof(uint64_t) * (nl ? nl : 1));
    uint32_t *xs = (uint32_t *)malloc(sizeof(uint32_t) * (nl ? nl : 1));
    uint32_t *tp = (uint32_t *)malloc(sizeof(uint32_t) * (nl ? nl : 1));
    uint32_t *tn = (uint32_t *)malloc(sizeof(uint32_t) * (nl ? nl : 1));
    uint32_t *sw = (uint32_t *)malloc(sizeof(uint32_t) * (nl ? nl : 1));
    uint32_t *held = (uint32_t *)malloc(sizeof(uint32_t) * (nl ? nl : 1));

    /* offset = lane % C; o = lane - offset + comb[offset] */
    for (uint64_t l = 0; l < nl; ++l) {
        uint64_t offset = l % C, base = l - offset;
        const uint8_t *c1, *c2;
        if (variant == ORC_VAR_BBS) {
            c1 = comb + (size_t)lanes[l].sel1 * C;
            c2 = comb + (size_t)(8 + lanes[l].sel2) * C;
        } else if (variant == ORC_VAR_BBS16) {
            /* chosen when the call starts, from BBS1's and BBS2's states */
            c1 = comb + (size_t)(lanes[l].y16[0] & 7u) * C;
            c2 = comb + (size_t)(8 + (lanes[l].y16[1] & 7u)) * C;
        } else {
            c1 = comb;
            c2 = comb + C;
        }
        p1[l] = base + c1[offset];
        p2[l] = base + c2[offset];
        xs[l] = lanes[l].x;
        tp[l] = lanes[l].tprev;
    }

    for (uint64_t i = 0; i < L; ++i) {
        for (uint64_t l = 0; l < nl; ++l) {
            if (variant == ORC_VAR_BBS) {
                orc_bbs_src s = {&lanes[l], NULL, 0};
                sw[l] = orc_bbs_strategy_src(&s, orc_bbs_w(lanes[l].M));
            } else if (variant == ORC_VAR_BBS16) {
                sw[l] = orc_bbs16_strategy(&lanes[l]);
            } else if (xl == ORC_XL_XOR128) {
                sw[l] = orc_xor128_step(lanes[l].w);
            } else if (xl == ORC_XL_XOR64) {
                uint64_t z = ((uint64_t)lanes[l].w[1] << 32) | lanes[l].w[0];
                z = orc_xor64_step(z);
                lanes[l].w[0] = (uint32_t)z;
                lanes[l].w[1] = (uint32_t)(z >> 32);
                sw[l] = (uint32_t)z;
            } else {
                lanes[l].w[0] = orc_xorshift32_step(lanes[l].w[0]);
                sw[l] = lanes[l].w[0];
            }
        }
        orc_mix_ci_iteration(nl, sw, p1, p2, tp, xs, tn);
        for (uint64_t l = 0; l < nl; ++l) {
            if (out)
                out[l * L + i] = xs[l];
            if (counts) {
                if ((i & 1) == 0) {
                    held[l] = xs[l];
                } else {
                    uint64_t a = held[l] >> 8, b = xs[l] >> 8;
                    if (a * a + b * b < (1ULL << 48))
                        counts[l] += 1;
                }
            }
        }
    }

    for (uint64_t l = 0; l < nl; ++l) {
        lanes[l].x = xs[l];
        lanes[l].tprev = tp[l];
        if (variant == ORC_VAR_BBS16 && L > 0)
            orc_bbs16_rotate(&lanes[l]);
    }
    free(p1);
    free(p2);
    free(xs);
    free(tp);
    free(tn);
    free(sw);
    free(held);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Chaotic Blum-Goldwasser (Sec. 9.2): Blum-Goldwasser whose keystream is    */
/* Eq. (Oplus) applied to the BBS bits, i.e. k_i = S0 ^ b_0 ^ ... ^ b_i.     */
/* ------------------------------------------------------------------------- */

static uint64_t orc_mulmod(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((unsigned __int128)a * b) % m);
}

static uint64_t orc_powmod(uint64_t a, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    a %= m;
    while (e) {
        if (e & 1)
            r = orc_mulmod(r, a, m);
        a = orc_mulmod(a, a, m);
        e >>= 1;
    }
    return r;
}

/* Inverse of a modulo m (gcd(a, m) = 1) by the extended Euclidean algorithm. */
static uint64_t orc_invmod(uint64_t a, uint64_t m)
{
    __int128 t = 0, nt = 1, r = (__int128)m, nr = (__int128)(a % m);
    while (nr != 0) {
        __int128 q = r / nr, tmp;
        tmp = t - q * nt; t = nt; nt = tmp;
        tmp = r - q * nr; r = nr; nr = tmp;
    }
    if (t < 0)
        t += m;
    return (uint64_t)t;
}

/* Encryption by Bob: x_0 = r^2 mod N; for i = 0 .. L-1: b_i = the w low bits
 * of x_i (w = floor(log2(floor(log2 N)))), c_i = m_i ^ (S0 ^ b_0 ^ ... ^ b_i),
 * x_{i+1} = x_i^2 mod N; the ciphertext is (c, y = x_L).  Returns w. */
uint32_t orc_bg_encrypt(uint64_t N, uint32_t S0, uint64_t r, uint64_t L, const uint8_t *m, uint8_t *c,
                        uint64_t *y)
{
    const uint32_t w = orc_bbs_w(N);
    const uint64_t mask = (1ULL << w) - 1;
    uint64_t x = orc_mulmod(r, r, N);
    uint32_t k = S0;
    for (uint64_t i = 0; i < L; ++i) {
        k ^= (uint32_t)(x & mask);
        c[i] = (uint8_t)(m[i] ^ k);
        x = orc_bbs_step(x, N);
    }
    *y = x;
    return w;
}

/* Alice's recovery of x_0 from y = x_0^(2^L) mod N with p = q = 3 mod 4:
 * r_p = y^(((p+1)/4)^L) mod p, r_q likewise (exponents reduced mod p - 1,
 * q - 1), x_0 = q (q^-1 mod p) r_p + p (p^-1 mod q) r_q mod N. */
uint64_t orc_bg_recover_x0(uint64_t p, uint64_t q, uint64_t y, uint64_t L)
{
    const uint64_t N = p * q;
    const uint64_t ep = orc_powmod((p + 1) / 4, L, p - 1);
    const uint64_t eq = orc_powmod((q + 1) / 4, L, q - 1);
    const uint64_t rp = orc_powmod(y % p, ep, p);
    const uint64_t rq = orc_powmod(y % q, eq, q);
    const uint64_t a = orc_mulmod(orc_mulmod(q, orc_invmod(q % p, p), N), rp, N);
    const uint64_t b = orc_mulmod(orc_mulmod(p, orc_invmod(p % q, q), N), rq, N);
    return (a + b) % N;
}

/* Decryption by Alice: recover x_0, regenerate b_i and the keystream
 * k_i = S0 ^ b_0 ^ ... ^ b_i, m_i = c_i ^ k_i. */
void orc_bg_decrypt(uint64_t p, uint64_t q, uint32_t S0, uint64_t y, uint64_t L, const uint8_t *c, uint8_t *m)
{
    const uint64_t N = p * q;
    const uint64_t mask = (1ULL << orc_bbs_w(N)) - 1;
    uint64_t x = orc_bg_recover_x0(p, q, y, L);
    uint32_t k = S0;
    for (uint64_t i = 0; i < L; ++i) {
        k ^= (uint32_t)(x & mask);
        m[i] = (uint8_t)(c[i] ^ k);
        x = orc_bbs_step(x, N);
    }
}

/* ------------------------------------------------------------------------- */
/* Listing 1 and Algorithm 3: the "naive" generator.  Each output XORs into   */
/* the 32-bit x the low and the high halves of one step of each of three      */
/* xor-like generators with 64-bit words: Marsaglia's xorshift with five      */
/* words (output (y + y + 1) v), xor128 (four words) and xorwow (five words   */
/* and a Weyl counter d += 362437, output d + v).  The paper names them and    */
/* cites Marsaglia's "Xorshift RNGs" without printing them; each recurrence   */
/* is written once, for a word type T, and the 32-bit instances (for which    */
/* Marsaglia chose the shifts: full periods 2^160 - 1 and 2^128 - 1) pin the  */
/* shift constants the 64-bit instances share.                                */
/* ------------------------------------------------------------------------- */

#define ORC_DEFINE_NAIVE_XORLIKES(T, SUF)                                      \
    T orc_xs160_step##SUF(T *s)                                                \
    {                                                                          \
        T t = s[0] ^ (s[0] >> 7);                                              \
        s[0] = s[1];                                                           \
        s[1] = s[2];                                                           \
        s[2] = s[3];                                                           \
        s[3] = s[4];                                                           \
        s[4] = (s[4] ^ (s[4] << 6)) ^ (t ^ (t << 13));                         \
        return (T)((T)(s[1] + s[1] + 1u) * s[4]);                              \
    }                                                                          \
    T orc_xor128w_step##SUF(T *s)                                              \
    {                                                                          \
        T t = s[0] ^ (s[0] << 11);                                             \
        s[0] = s[1];                                                           \
        s[1] = s[2];                                                           \
        s[2] = s[3];                                                           \
        s[3] = (s[3] ^ (s[3] >> 19)) ^ (t ^ (t >> 8));                         \
        return s[3];                                                           \
    }                                                                          \
    T orc_xorwow_step##SUF(T *s, T *d)                                         \
    {                                                                          \
        T t = s[0] ^ (s[0] >> 2);                                              \
        s[0] = s[1];                                                           \
        s[1] = s[2];                                                           \
        s[2] = s[3];                                                           \
        s[3] = s[4];                                                           \
        s[4] = (s[4] ^ (s[4] << 4)) ^ (t ^ (t << 1));                          \
        *d = (T)(*d + 362437u);                                                \
        return (T)(*d + s[4]);                                                 \
    }

ORC_DEFINE_NAIVE_XORLIKES(uint32_t, 32)
ORC_DEFINE_NAIVE_XORLIKES(uint64_t, 64)

/* Listing 1 (Sec. 5) XORs into x the low and the high 32-bit half of each of
 * t1, t2 and t3.  XOR is associative and commutative, so that is x XOR the two
 * halves of T = t1 XOR t2 XOR t3. */
uint32_t orc_listing1_combine(uint32_t x, uint64_t t1, uint64_t t2, uint64_t t3)
{
    const uint64_t T = t1 ^ t2 ^ t3;
    return x ^ (uint32_t)T ^ (uint32_t)(T >> 32);
}

typedef struct {
    uint64_t xs[5];   /* xorshift (five words) */
    uint64_t xo[4];   /* xor128                */
    uint64_t xw[5];   /* xorwow                */
    uint64_t d;       /* xorwow's Weyl counter */
    uint32_t x;       /* the CI state          */
    uint32_t pad;
} orc_naive_lane;

uint32_t orc_naive_lane_size(void) { return (uint32_t)sizeof(orc_naive_lane); }

static uint32_t orc_naive_next(orc_naive_lane *L)
{
    const uint64_t t1 = orc_xs160_step64(L->xs);
    const uint64_t t2 = orc_xor128w_step64(L->xo);
    const uint64_t t3 = orc_xorwow_step64(L->xw, &L->d);
    L->x = orc_listing1_combine(L->x, t1, t2, t3);
    return L->x;
}

/* Listing 1 as a sequential program: the CI state starts at x0 and the three
 * xor-likes at the start words of Marsaglia's published generators (x, y, z, w,
 * v = 123456789, 362436069, 521288629, 88675123, 5783321; d = 6615241). */
void orc_listing1_run(uint32_t x0, uint64_t n, uint32_t *out)
{
    orc_naive_lane L;
    const uint64_t seeds[5] = {123456789u, 362436069u, 521288629u, 88675123u, 5783321u};
    for (int i = 0; i < 5; ++i) {
        L.xs[i] = seeds[i];
        L.xw[i] = seeds[i];
    }
    for (int i = 0; i < 4; ++i) L.xo[i] = seeds[i];
    L.d = 6615241u;
    L.x = x0;
    for (uint64_t i = 0; i < n; ++i) out[i] = orc_naive_next(&L);
}

/* Algorithm 3's per-thread parameters (ISAAC on the host in the paper; the
 * counter-based splitmix64 draws here): lane s takes draws 0-4 for the
 * xorshift words, 5-8 for xor128, 9-13 for xorwow, 14 for d and the low half
 * of 15 for x.  An all-zero word set (never drawn in practice) becomes 1, 0, ... */
void orc_naive_init_lanes(uint64_t seed, uint64_t lane0, uint64_t nl, orc_naive_lane *lanes)
{
    for (uint64_t i = 0; i < nl; ++i) {
        orc_naive_lane *L = &lanes[i];
        const uint64_t s = lane0 + i;
        uint64_t k = 0, any;
        any = 0;
        for (int w = 0; w < 5; ++w) any |= (L->xs[w] = orc_lane_draw(seed, s, k++));
        if (!any) L->xs[0] = 1;
        any = 0;
        for (int w = 0; w < 4; ++w) any |= (L->xo[w] = orc_lane_draw(seed, s, k++));
        if (!any) L->xo[0] = 1;
        any = 0;
        for (int w = 0; w < 5; ++w) any |= (L->xw[w] = orc_lane_draw(seed, s, k++));
        if (!any) L->xw[0] = 1;
        L->d = orc_lane_draw(seed, s, k++);
        L->x = (uint32_t)orc_lane_draw(seed, s, k++);
        L->pad = 0;
    }
}

/* Algorithm 3: every lane (thread) runs Listing 1 on its own state, with no
 * exchange between lanes; out[l * n + i] is lane l's (i + 1)-th output. */
void orc_naive_run(orc_naive_lane *lanes, uint64_t nl, uint64_t n, uint32_t *out)
{
    for (uint64_t l = 0; l < nl; ++l)
        for (uint64_t i = 0; i < n; ++i) {
            const uint32_t v = orc_naive_next(&lanes[l]);
            if (out) out[l * n + i] = v;
        }
}
