/*
 * Oracle for Hissoiny, Despres & Ozell, "Using graphics processing units to
 * generate random numbers" (arXiv:1101.1846).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded C that writes the
 * paper's recurrences out literally, one stream and one step at a time, with
 * no blocking, unrolling or reordering.  Only tests/, __graft_entry__.smoke()
 * and bench.py's CPU baseline / reference arm may load it.  It shares no code
 * with the CUDA library.
 *
 * Parity status of each part (what pins it is in tests/test_oracle_pins.py and
 * tests/test_oracle_seeding.py):
 *   primality, multiplier search ... pinned (392 count of Sec. "Methods /
 *                                    multiply-with-carry"; brute force)
 *   MWC step ....................... pinned (Lehmer closed form; periods)
 *   xor128 step .................... pinned (full period 2^128-1 over GF(2))
 *   xorshift32 step ................ pinned (period 2^32-1); its shift ORDER
 *                                    is parity unpinned (both orders of Eq. 6
 *                                    have full period)
 *   LCG step ....................... pinned (Eq. 7 constants; period 2^32)
 *   KISS combination ............... pinned (sum of independently stepped parts)
 *   FP32 uniform ................... pinned (exactness, range)
 *   splitmix64 ..................... pinned (increment = golden ratio;
 *                                    published outputs from three states)
 *   seeding, every kind ............ pinned (the draw-to-state mapping
 *                                    restated with Python integers; each
 *                                    redraw branch reached by a seed found by
 *                                    inverting the finaliser)
 *   consumers (sums, disc count) ... pinned (closed-form sums of synthetic
 *                                    sequences; lattice count of the quarter
 *                                    disc by integer square roots)
 *   jump-ahead ..................... pinned (equal to stepping; periods of
 *                                    each part reached by one jump)
 *   the paper's own generators:
 *     two-part base-2^16 MWC ....... pinned (parts are the pinned base-2^16
 *                                    step; Lehmer closed form of the joined
 *                                    output; pairs in lexicographic order);
 *                                    joining by + rather than | is the reading
 *                                    the paper's operation count fixes
 *     r = 8 XorShift (Eq. 5) ....... pinned (period 2^256-1 over GF(2); the
 *                                    five lags); the order of the factors of
 *                                    (I+L^24)(I+R^7) is parity unpinned: both
 *                                    orders have full period
 *     KISS, xor form ............... pinned (parts stepped on their own)
 *   battery counts ................. pinned (closed-form counts of synthetic
 *                                    outputs; birthday samples built from
 *                                    spacing lists with known repeats)
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Number theory for the multiplier condition (Sec. "multiply-with-carry"
 * of the background: a*b-1 must be a safe prime).                        */
/* ------------------------------------------------------------------ */

uint64_t oracle_mulmod_u64(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((unsigned __int128)a * b) % m);
}

uint64_t oracle_powmod_u64(uint64_t base, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    base %= m;
    while (e) {
        if (e & 1)
            r = oracle_mulmod_u64(r, base, m);
        base = oracle_mulmod_u64(base, base, m);
        e >>= 1;
    }
    return r;
}

/* Odd primes below 1024, by a sieve of Eratosthenes on first use. */
static int g_small_primes[200];
static int g_n_small_primes = 0;

static void init_small_primes(void)
{
    if (g_n_small_primes)
        return;
    char composite[1024] = {0};
    int n = 0;
    for (int i = 3; i < 1024; i += 2) {
        if (composite[i])
            continue;
        g_small_primes[n++] = i;
        for (int j = i * i; j < 1024; j += 2 * i)
            composite[j] = 1;
    }
    g_n_small_primes = n;
}

/* Trial division by 2 and the odd primes below 1024: returns 0 when n is
 * composite (or < 2), 1 when n is proven prime (n < 1024^2 with no factor
 * found), 2 when undecided. */
static int small_factor_test(uint64_t n)
{
    init_small_primes();
    if (n < 2)
        return 0;
    if (n % 2 == 0)
        return n == 2;
    for (int i = 0; i < g_n_small_primes; ++i) {
        uint64_t l = (uint64_t)g_small_primes[i];
        if (n % l == 0)
            return n == l;
    }
    return n < 1024ull * 1024ull ? 1 : 2;
}

/* Deterministic Miller-Rabin for every n < 2^64: the first twelve primes as
 * bases are a proven deterministic set below 3.3e24 (Sorenson and Webster,
 * "Strong pseudoprimes to twelve prime bases", Math. Comp. 2017).  n must be
 * odd and larger than 37. */
static const uint64_t k_mr_bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};

static int miller_rabin(uint64_t n)
{
    /* n - 1 = d * 2^r with d odd */
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) {
        d >>= 1;
        ++r;
    }
    for (int i = 0; i < 12; ++i) {
        uint64_t x = oracle_powmod_u64(k_mr_bases[i], d, n);
        if (x == 1 || x == n - 1)
            continue;
        int witness = 1;
        for (int k = 1; k < r; ++k) {
            x = oracle_mulmod_u64(x, x, n);
            if (x == n - 1) {
                witness = 0;
                break;
            }
        }
        if (witness)
            return 0;
    }
    return 1;
}

int oracle_is_prime_u64(uint64_t n)
{
    int v = small_factor_test(n);
    if (v != 2)
        return v;
    return miller_rabin(n);
}

/* The multiplier condition: p = a*b - 1 is a safe prime, i.e. p and
 * (p - 1)/2 are both prime, with b = 2^log2b.  Both numbers are trial
 * divided before either gets the slower Miller-Rabin test; the verdict is
 * the same as oracle_is_prime_u64(q) && oracle_is_prime_u64(p). */
int oracle_is_safe_multiplier(uint64_t a, int log2b)
{
    if (a == 0)
        return 0;
    uint64_t p = a * ((uint64_t)1 << log2b) - 1;
    uint64_t q = (p - 1) / 2;
    int vq = small_factor_test(q);
    if (vq == 0)
        return 0;
    int vp = small_factor_test(p);
    if (vp == 0)
        return 0;
    return (vq == 1 || miller_rabin(q)) && (vp == 1 || miller_rabin(p));
}

/* The first k valid multipliers scanning a = a_top, a_top - 1, ..., 1.
 * Returns how many were found (k unless the scan reached a = 0). */
uint64_t oracle_multipliers(int log2b, uint64_t a_top, uint64_t k, uint32_t *out)
{
    uint64_t found = 0;
    for (uint64_t a = a_top; a >= 1 && found < k; --a) {
        if (oracle_is_safe_multiplier(a, log2b))
            out[found++] = (uint32_t)a;
    }
    return found;
}

/* Every valid multiplier in [a_lo, a_hi], in descending order.  Returns the
 * count; only the first `cap` are written.  Consecutive ranges concatenate
 * to the same list oracle_multipliers produces. */
uint64_t oracle_multipliers_range(int log2b, uint64_t a_hi, uint64_t a_lo,
                                  uint32_t *out, uint64_t cap)
{
    uint64_t found = 0;
    if (a_lo < 1)
        a_lo = 1;
    for (uint64_t a = a_hi; a >= a_lo; --a) {
        if (oracle_is_safe_multiplier(a, log2b)) {
            if (found < cap)
                out[found] = (uint32_t)a;
            ++found;
        }
        if (a == a_lo)
            break;
    }
    return found;
}

/* Multiplier pairs of the paper's two-part MWC: the first k pairs (i, j),
 * i < j, of the 392 base-2^16 multipliers (largest first) in lexicographic
 * order, packed as table[i] | table[j] << 16 (parametrisation by pairs of
 * multipliers, Methods / MWC).  Returns how many were written (at most
 * 392 * 391 / 2). */
uint64_t oracle_mwc16_pairs(uint64_t k, uint32_t *out)
{
    uint32_t table[512];
    uint64_t m = oracle_multipliers(16, 0xFFFF, 512, table);
    uint64_t found = 0;
    for (uint64_t i = 0; i < m && found < k; ++i)
        for (uint64_t j = i + 1; j < m && found < k; ++j)
            out[found++] = table[i] | (table[j] << 16);
    return found;
}

/* ------------------------------------------------------------------ */
/* Seeding.  The paper gives every thread its own seeds (parametrisation,
 * Sec. "Parallelizing RNGs" and the MWC/KISS kernel descriptions) without
 * saying how they are made; they are drawn here from splitmix64 (Steele,
 * Lea and Flood, "Fast splittable pseudorandom number generators", 2014)
 * started at seed + stream index.                                       */
/* ------------------------------------------------------------------ */

uint64_t oracle_splitmix64(uint64_t *z)
{
    *z += 0x9E3779B97F4A7C15ull;
    uint64_t r = *z;
    r = (r ^ (r >> 30)) * 0xBF58476D1CE4E5B9ull;
    r = (r ^ (r >> 27)) * 0x94D049BB133111EBull;
    return r ^ (r >> 31);
}

static uint32_t lo32(uint64_t v) { return (uint32_t)(v & 0xFFFFFFFFull); }
static uint32_t hi32(uint64_t v) { return (uint32_t)(v >> 32); }

/* MWC (x, c) from successive draws: c is reduced below a so that the state
 * is one of the Lehmer-form states, and the two fixed points (0, 0) and
 * (b - 1, a - 1) are skipped by drawing again. */
static void seed_mwc(uint32_t a, uint64_t *z, uint32_t *x, uint32_t *c)
{
    for (;;) {
        uint64_t r = oracle_splitmix64(z);
        *x = lo32(r);
        *c = hi32(r) % a;
        int zero = (*x == 0 && *c == 0);
        int top = (*x == 0xFFFFFFFFu && *c == a - 1);
        if (!zero && !top)
            return;
    }
}

/* The paper's MWC pair from one draw: (x, c) of the first part from bits
 * 0-15 and 16-31 (c reduced below a1), of the second from bits 32-47 and
 * 48-63 (c below a2); drawn again while either part is a fixed point. */
static void seed_mwc16x2(uint32_t a_pair, uint64_t *z, uint32_t *zw)
{
    uint32_t a1 = a_pair & 0xFFFFu, a2 = a_pair >> 16;
    for (;;) {
        uint64_t r = oracle_splitmix64(z);
        uint32_t x1 = (uint32_t)(r & 0xFFFFu), c1 = (uint32_t)((r >> 16) & 0xFFFFu) % a1;
        uint32_t x2 = (uint32_t)((r >> 32) & 0xFFFFu), c2 = (uint32_t)(r >> 48) % a2;
        int bad1 = (x1 == 0 && c1 == 0) || (x1 == 0xFFFFu && c1 == a1 - 1);
        int bad2 = (x2 == 0 && c2 == 0) || (x2 == 0xFFFFu && c2 == a2 - 1);
        if (!bad1 && !bad2) {
            zw[0] = x1 | (c1 << 16);
            zw[1] = x2 | (c2 << 16);
            return;
        }
    }
}

void oracle_seed_stream(int kind, uint32_t a, uint64_t seed, uint64_t s,
                        uint32_t *st)
{
    uint64_t z = seed + s;
    memset(st, 0, (size_t)oracle_state_words(kind) * sizeof(uint32_t));
    if (kind == 3) {
        seed_mwc16x2(a, &z, st);
        return;
    }
    if (kind == 4) {
        for (;;) {
            uint32_t any = 0;
            for (int i = 0; i < 4; ++i) {
                uint64_t r = oracle_splitmix64(&z);
                st[2 * i] = lo32(r);
                st[2 * i + 1] = hi32(r);
                any |= st[2 * i] | st[2 * i + 1];
            }
            if (any)
                return;
        }
    }
    if (kind == 5) {
        seed_mwc16x2(a, &z, st);
        uint64_t r = oracle_splitmix64(&z);
        st[2] = lo32(r);
        st[3] = hi32(r);
        while (st[2] == 0)
            st[2] = lo32(oracle_splitmix64(&z));
        return;
    }
    if (kind == 0) {
        seed_mwc(a, &z, &st[0], &st[1]);
    } else if (kind == 1) {
        for (;;) {
            uint64_t r0 = oracle_splitmix64(&z);
            uint64_t r1 = oracle_splitmix64(&z);
            st[0] = lo32(r0);
            st[1] = hi32(r0);
            st[2] = lo32(r1);
            st[3] = hi32(r1);
            if (st[0] | st[1] | st[2] | st[3])
                return;
        }
    } else {
        seed_mwc(a, &z, &st[0], &st[1]);
        uint64_t r = oracle_splitmix64(&z);
        st[2] = lo32(r);
        st[3] = hi32(r);
        while (st[2] == 0)
            st[2] = lo32(oracle_splitmix64(&z));
    }
}

/* ------------------------------------------------------------------ */
/* The generators.                                                      */
/* ------------------------------------------------------------------ */

/* Eq. 2-3: x_{n+1} = (a x_n + c_n) mod b, c_{n+1} = floor((a x_n + c_n)/b),
 * written with the division and remainder themselves; b = 2^log2b. */
uint32_t oracle_mwc_step(uint32_t a, uint32_t *x, uint32_t *c, int log2b)
{
    uint64_t b = (uint64_t)1 << log2b;
    uint64_t t = (uint64_t)a * (uint64_t)(*x) + (uint64_t)(*c);
    *x = (uint32_t)(t % b);
    *c = (uint32_t)(t / b);
    return *x;
}

/* xor128 (Marsaglia, "Xorshift RNGs", J. Stat. Softw. 8(14), 2003): state
 * (x, y, z, w); t = x ^ (x << 11); the words shift down by one; the new w is
 * w ^ (w >> 19) ^ t ^ (t >> 8), which is also the output. */
uint32_t oracle_xor128_step(uint32_t st[4])
{
    uint32_t x = st[0];
    uint32_t t = x ^ (x << 11);
    st[0] = st[1];
    st[1] = st[2];
    st[2] = st[3];
    uint32_t w = st[3];
    st[3] = w ^ (w >> 19) ^ t ^ (t >> 8);
    return st[3];
}

/* Eq. 6: the type-I xorshift with A1 = (I + L^13)(I + R^17)(I + L^5),
 * applied as <<13, then >>17, then <<5. */
uint32_t oracle_xorshift32_step(uint32_t *y)
{
    uint32_t v = *y;
    v ^= v << 13;
    v ^= v >> 17;
    v ^= v << 5;
    *y = v;
    return v;
}

/* Eq. 7 with a = 69069, c = 1234567, m = 2^32. */
uint32_t oracle_lcg_step(uint32_t *z)
{
    uint64_t m = (uint64_t)1 << 32;
    *z = (uint32_t)((69069ull * (uint64_t)(*z) + 1234567ull) % m);
    return *z;
}

/* KISS: each of the three parts advances once and the output is the sum of
 * their new values mod 2^32. */
uint32_t oracle_kiss_step(uint32_t a, uint32_t st[4])
{
    uint32_t m = oracle_mwc_step(a, &st[0], &st[1], 32);
    uint32_t y = oracle_xorshift32_step(&st[2]);
    uint32_t z = oracle_lcg_step(&st[3]);
    return (uint32_t)(((uint64_t)m + y + z) % ((uint64_t)1 << 32));
}

/* The paper's own MWC (Methods, "multiply-with-carry"): two base-2^16
 * MWCs with 16-bit multipliers a1 = a_pair & 0xFFFF and a2 = a_pair >> 16.
 * Each is kept in one 32-bit word z = x + c 2^16 (x the last value, c the
 * carry); one step of Eq. 2-3 with b = 2^16 maps it to a (z mod 2^16) +
 * (z div 2^16).  The output joins the two new words as (z << 16) + w mod
 * 2^32: three shifts, two ands, two multiplies and three adds, the
 * operation count the paper gives for its loop. */
uint32_t oracle_mwc16x2_step(uint32_t a_pair, uint32_t st[2])
{
    uint32_t a1 = a_pair & 0xFFFFu, a2 = a_pair >> 16;
    uint32_t x = st[0] & 0xFFFFu, c = st[0] >> 16;
    oracle_mwc_step(a1, &x, &c, 16);
    st[0] = x | (c << 16);
    x = st[1] & 0xFFFFu;
    c = st[1] >> 16;
    oracle_mwc_step(a2, &x, &c, 16);
    st[1] = x | (c << 16);
    return (uint32_t)((((uint64_t)st[0] << 16) + st[1]) % ((uint64_t)1 << 32));
}

/* Eq. 5, Panneton's XorShift with r = 8 words and s = 7 xorshifts:
 * st = (v_{n-8}, ..., v_{n-1});
 *   v_n = (I+L^9)(I+L^13) v_{n-1} + (I+L^7) v_{n-4} + (I+R^3) v_{n-5}
 *       + (I+R^10) v_{n-7} + (I+L^24)(I+R^7) v_{n-8}
 * over GF(2) (+ is xor), each product applied right to left as in Eq. 4's
 * v_i = sum A_j v_{i-j}; the words shift down and v_n, the output, enters
 * at the top. */
uint32_t oracle_xorshift8_step(uint32_t st[8])
{
    uint32_t t1 = st[7] ^ (st[7] << 13);
    t1 ^= t1 << 9;
    uint32_t t4 = st[4] ^ (st[4] << 7);
    uint32_t t5 = st[3] ^ (st[3] >> 3);
    uint32_t t7 = st[1] ^ (st[1] >> 10);
    uint32_t t8 = st[0] ^ (st[0] >> 7);
    t8 ^= t8 << 24;
    uint32_t v = t1 ^ t4 ^ t5 ^ t7 ^ t8;
    for (int i = 0; i < 7; ++i)
        st[i] = st[i + 1];
    st[7] = v;
    return v;
}

/* KISS as the paper's Background section combines it: the MWC and LCG
 * values are xored and the XorShift value is added, with the paper's own
 * two-part MWC: ((MWC xor LCG) + xorshift32) mod 2^32.  State {z, w, y, z_lcg}. */
uint32_t oracle_kiss_xor_step(uint32_t a_pair, uint32_t st[4])
{
    uint32_t m = oracle_mwc16x2_step(a_pair, st);
    uint32_t y = oracle_xorshift32_step(&st[2]);
    uint32_t z = oracle_lcg_step(&st[3]);
    return (uint32_t)(((uint64_t)(m ^ z) + y) % ((uint64_t)1 << 32));
}

uint32_t oracle_step(int kind, uint32_t a, uint32_t *st)
{
    if (kind == 0)
        return oracle_mwc_step(a, &st[0], &st[1], 32);
    if (kind == 1)
        return oracle_xor128_step(st);
    if (kind == 2)
        return oracle_kiss_step(a, st);
    if (kind == 3)
        return oracle_mwc16x2_step(a, st);
    if (kind == 4)
        return oracle_xorshift8_step(st);
    return oracle_kiss_xor_step(a, st);
}

int oracle_state_words(int kind) { return kind == 4 ? 8 : 4; }

/* Uniform in [0, 1): the top 24 bits of u as an integer times 2^-24.  Both
 * the conversion (a 24-bit integer) and the power-of-two scaling are exact
 * in binary32. */
float oracle_to_unit_f32(uint32_t u)
{
    return (float)(u >> 8) * (1.0f / 16777216.0f);
}

/* One stream: n outputs written contiguously, state advanced in place. */
void oracle_stream(int kind, uint32_t a, uint32_t *st, uint64_t n, int fmt,
                   void *out)
{
    for (uint64_t j = 0; j < n; ++j) {
        uint32_t u = oracle_step(kind, a, st);
        if (fmt == 0)
            ((uint32_t *)out)[j] = u;
        else
            ((float *)out)[j] = oracle_to_unit_f32(u);
    }
}

/* One generate call over all streams: output j of stream s goes to
 * out[j * n_streams + s]; state holds W = oracle_state_words(kind) words per
 * stream (st[W*s + w]). */
void oracle_generate(int kind, uint64_t n_streams, const uint32_t *a,
                     uint32_t *state, uint64_t n_per_stream, int fmt,
                     void *out)
{
    for (uint64_t s = 0; s < n_streams; ++s) {
        uint32_t *st = state + (uint64_t)oracle_state_words(kind) * s;
        uint32_t as = a ? a[s] : 0;
        for (uint64_t j = 0; j < n_per_stream; ++j) {
            uint32_t u = oracle_step(kind, as, st);
            uint64_t idx = j * n_streams + s;
            if (fmt == 0)
                ((uint32_t *)out)[idx] = u;
            else
                ((float *)out)[idx] = oracle_to_unit_f32(u);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Brute-force periods.                                                 */
/* ------------------------------------------------------------------ */

/* Steps until (x, c) returns to (x0, c0); 0 if not within `limit` steps. */
uint64_t oracle_mwc_period(uint32_t a, uint32_t x0, uint32_t c0, int log2b,
                           uint64_t limit)
{
    uint32_t x = x0, c = c0;
    for (uint64_t n = 1; n <= limit; ++n) {
        oracle_mwc_step(a, &x, &c, log2b);
        if (x == x0 && c == c0)
            return n;
    }
    return 0;
}

uint64_t oracle_xorshift32_period(uint32_t y0)
{
    uint32_t y = y0;
    uint64_t n = 0;
    do {
        oracle_xorshift32_step(&y);
        ++n;
    } while (y != y0 && n <= 0x100000000ull);
    return n;
}

uint64_t oracle_lcg_period(uint32_t z0)
{
    uint32_t z = z0;
    uint64_t n = 0;
    do {
        oracle_lcg_step(&z);
        ++n;
    } while (z != z0 && n <= 0x100000001ull);
    return n;
}

/* ------------------------------------------------------------------ */
/* Batch helpers for the Python wrapper (loops over the functions above). */
/* ------------------------------------------------------------------ */

/* Seeds the streams listed in s_ids (n of them); a[i] is the multiplier of
 * stream s_ids[i] (ignored for xor128); st receives 4 words per stream. */
void oracle_seed_streams(int kind, const uint32_t *a, uint64_t seed,
                         const uint64_t *s_ids, uint64_t n, uint32_t *st)
{
    for (uint64_t i = 0; i < n; ++i)
        oracle_seed_stream(kind, a ? a[i] : 0, seed, s_ids[i],
                           st + (uint64_t)oracle_state_words(kind) * i);
}

/* ------------------------------------------------------------------ */
/* Consumers with no output array.  The paper also times its generators
 * with the numbers kept on chip and only the final state stored, the case
 * of an application that calls the generator inline (Sec. "Performance
 * evaluation"; the "without writeback" rows of Tables I-III).  Here each
 * consumer reads one stream's outputs in order and reduces them to one
 * 64-bit number, so that every output is used.                          */
/* ------------------------------------------------------------------ */

/* Sum of the outputs, mod 2^64. */
uint64_t oracle_sum_u32(const uint32_t *u, uint64_t n)
{
    uint64_t s = 0;
    for (uint64_t j = 0; j < n; ++j)
        s += (uint64_t)u[j];
    return s;
}

/* Sum of the 24-bit integers u >> 8: exactly 2^24 times the sum of the
 * float32 uniforms of the same outputs. */
uint64_t oracle_sum_u24(const uint32_t *u, uint64_t n)
{
    uint64_t s = 0;
    for (uint64_t j = 0; j < n; ++j)
        s += (uint64_t)(u[j] >> 8);
    return s;
}

/* Consecutive outputs taken two at a time, (u[2k], u[2k+1]) for
 * k < floor(n / 2), as the point (x, y) of their float32 uniforms: the
 * number of points with x^2 + y^2 < 1.  With x = X 2^-24 and y = Y 2^-24
 * the test is X^2 + Y^2 < 2^48, evaluated exactly in integers.  The count
 * over P points estimates P pi / 4. */
uint64_t oracle_disc_count(const uint32_t *u, uint64_t n)
{
    uint64_t inside = 0;
    for (uint64_t k = 0; 2 * k + 1 < n; ++k) {
        uint64_t X = u[2 * k] >> 8;
        uint64_t Y = u[2 * k + 1] >> 8;
        if (X * X + Y * Y < ((uint64_t)1 << 48))
            ++inside;
    }
    return inside;
}

/* Every stream advances n_per_stream steps (state in place, laid out as in
 * oracle_generate); out[s] is the chosen consumer applied to
 * stream s's outputs: op 0 = oracle_sum_u32, 1 = oracle_sum_u24,
 * 2 = oracle_disc_count.  Returns 0, or -1 if the scratch row cannot be
 * allocated. */
int oracle_reduce(int kind, uint64_t n_streams, const uint32_t *a,
                  uint32_t *state, uint64_t n_per_stream, int op,
                  uint64_t *out)
{
    uint32_t *row = (uint32_t *)malloc((n_per_stream ? n_per_stream : 1) * sizeof(uint32_t));
    if (!row)
        return -1;
    for (uint64_t s = 0; s < n_streams; ++s) {
        oracle_stream(kind, a ? a[s] : 0, state + (uint64_t)oracle_state_words(kind) * s,
                      n_per_stream, 0, row);
        if (op == 0)
            out[s] = oracle_sum_u32(row, n_per_stream);
        else if (op == 1)
            out[s] = oracle_sum_u24(row, n_per_stream);
        else
            out[s] = oracle_disc_count(row, n_per_stream);
    }
    free(row);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Jump-ahead: the state k steps later, computed without the steps in
 * between.  Sequence splitting needs it (Sec. "Parallelizing RNGs": a
 * node starts where the previous node's block of numbers ends).          */
/* ------------------------------------------------------------------ */

/* MWC, b = 2^log2b, p = a b - 1.  With t = a x + c (0 < t < p for every
 * state except the two fixed points), one step gives
 *   x' = t mod b,  c' = t div b,  t' = a x' + c',
 * and b t' = a b (t mod b) + t - (t mod b) = t + p (t mod b), so
 * t' = b^-1 t = a t (mod p) because a b = 1 (mod p).  Hence k steps
 * multiply t by a^k mod p, and (x, c) is recovered from t as
 * x = t div a, c = t mod a (the state keeps 0 <= c < a). */
void oracle_mwc_jump(uint32_t a, uint32_t *x, uint32_t *c, uint64_t k,
                     int log2b)
{
    uint64_t p = (uint64_t)a * ((uint64_t)1 << log2b) - 1;
    uint64_t t = (uint64_t)(*c) + (uint64_t)(*x) * a;
    t = oracle_mulmod_u64(oracle_powmod_u64(a, k, p), t, p);
    *x = (uint32_t)(t / a);
    *c = (uint32_t)(t % a);
}

/* GF(2) matrices of at most 128 x 128 bits.  Bit i of a state vector is
 * bit (i mod 32) of word i / 32.  Column j of the matrix of a linear step
 * is the image of the unit vector e_j under the step. */
typedef struct {
    int nbits;
    uint32_t col[256][8];
} gf2mat;

static void gf2_apply(const gf2mat *m, const uint32_t v[8], uint32_t out[8])
{
    uint32_t r[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int j = 0; j < m->nbits; ++j) {
        if ((v[j / 32] >> (j % 32)) & 1u) {
            for (int w = 0; w < 8; ++w)
                r[w] ^= m->col[j][w];
        }
    }
    memcpy(out, r, (size_t)((m->nbits + 31) / 32) * sizeof(uint32_t));
}

/* out = a * b: column j of the product is a applied to column j of b. */
static void gf2_mul(const gf2mat *a, const gf2mat *b, gf2mat *out)
{
    gf2mat r;
    memset(&r, 0, sizeof(r));
    r.nbits = a->nbits;
    for (int j = 0; j < a->nbits; ++j)
        gf2_apply(a, b->col[j], r.col[j]);
    *out = r;
}

static void gf2_identity(gf2mat *m, int nbits)
{
    memset(m, 0, sizeof(*m));
    m->nbits = nbits;
    for (int j = 0; j < nbits; ++j)
        m->col[j][j / 32] = 1u << (j % 32);
}

/* m^k by binary powering. */
static void gf2_pow(const gf2mat *m, uint64_t k, gf2mat *out)
{
    gf2mat result, base = *m;
    gf2_identity(&result, m->nbits);
    while (k) {
        if (k & 1)
            gf2_mul(&result, &base, &result);
        gf2_mul(&base, &base, &base);
        k >>= 1;
    }
    *out = result;
}

static void xor128_matrix(gf2mat *m)
{
    memset(m, 0, sizeof(*m));
    m->nbits = 128;
    for (int j = 0; j < 128; ++j) {
        uint32_t st[4] = {0, 0, 0, 0};
        st[j / 32] = 1u << (j % 32);
        oracle_xor128_step(st);
        memcpy(m->col[j], st, sizeof(st));
    }
}

static void xorshift8_matrix(gf2mat *m)
{
    memset(m, 0, sizeof(*m));
    m->nbits = 256;
    for (int j = 0; j < 256; ++j) {
        uint32_t st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        st[j / 32] = 1u << (j % 32);
        oracle_xorshift8_step(st);
        memcpy(m->col[j], st, sizeof(st));
    }
}

static void xorshift32_matrix(gf2mat *m)
{
    memset(m, 0, sizeof(*m));
    m->nbits = 32;
    for (int j = 0; j < 32; ++j) {
        uint32_t y = 1u << j;
        oracle_xorshift32_step(&y);
        m->col[j][0] = y;
    }
}

/* The matrices are large (8 KB each): kept in static storage. */
static gf2mat g_m, g_mk;

void oracle_xor128_jump(uint32_t st[4], uint64_t k)
{
    uint32_t v[8] = {st[0], st[1], st[2], st[3], 0, 0, 0, 0};
    xor128_matrix(&g_m);
    gf2_pow(&g_m, k, &g_mk);
    gf2_apply(&g_mk, v, v);
    memcpy(st, v, 4 * sizeof(uint32_t));
}

void oracle_xorshift32_jump(uint32_t *y, uint64_t k)
{
    uint32_t v[8] = {*y, 0, 0, 0, 0, 0, 0, 0};
    xorshift32_matrix(&g_m);
    gf2_pow(&g_m, k, &g_mk);
    gf2_apply(&g_mk, v, v);
    *y = v[0];
}

void oracle_xorshift8_jump(uint32_t st[8], uint64_t k)
{
    xorshift8_matrix(&g_m);
    gf2_pow(&g_m, k, &g_mk);
    gf2_apply(&g_mk, st, st);
}

/* Eq. 7's map z -> A z + C (mod 2^32) applied k times.  Two affine maps
 * compose as (A1, C1) after (A2, C2) = (A1 A2, A1 C2 + C1). */
void oracle_lcg_jump(uint32_t *z, uint64_t k)
{
    uint64_t m = (uint64_t)1 << 32;
    uint64_t RA = 1, RC = 0;              /* result: the identity map */
    uint64_t BA = 69069, BC = 1234567;    /* base: one step */
    while (k) {
        if (k & 1) {
            RC = (BA * RC + BC) % m;      /* base after result */
            RA = (BA * RA) % m;
        }
        BC = (BA * BC + BC) % m;          /* base after base */
        BA = (BA * BA) % m;
        k >>= 1;
    }
    *z = (uint32_t)((RA * (uint64_t)(*z) + RC) % m);
}

/* One base-2^16 MWC packed as x | c << 16 (see oracle_mwc16x2_step). */
static void mwc16_jump(uint32_t a, uint32_t *z, uint64_t k)
{
    uint32_t x = *z & 0xFFFFu, c = *z >> 16;
    oracle_mwc_jump(a, &x, &c, k, 16);
    *z = x | (c << 16);
}

void oracle_jump(int kind, uint32_t a, uint32_t *st, uint64_t k)
{
    if (kind == 0) {
        oracle_mwc_jump(a, &st[0], &st[1], k, 32);
    } else if (kind == 1) {
        oracle_xor128_jump(st, k);
    } else if (kind == 2) {
        oracle_mwc_jump(a, &st[0], &st[1], k, 32);
        oracle_xorshift32_jump(&st[2], k);
        oracle_lcg_jump(&st[3], k);
    } else if (kind == 3) {
        mwc16_jump(a & 0xFFFFu, &st[0], k);
        mwc16_jump(a >> 16, &st[1], k);
    } else if (kind == 4) {
        oracle_xorshift8_jump(st, k);
    } else {
        mwc16_jump(a & 0xFFFFu, &st[0], k);
        mwc16_jump(a >> 16, &st[1], k);
        oracle_xorshift32_jump(&st[2], k);
        oracle_lcg_jump(&st[3], k);
    }
}

/* ------------------------------------------------------------------ */
/* A small statistical battery: counts over a block of outputs u laid out
 * stream-interleaved (u[j * n_streams + s], j < n_per_stream).  The paper
 * assesses its generators with DIEHARD and TestU01 (Sec. "Performance
 * evaluation"); these are four tests of those families, written from their
 * definitions; the statistics and p-values are formed from the counts.  */
/* ------------------------------------------------------------------ */

/* Monobit: the number of one bits in all outputs. */
uint64_t oracle_bat_ones(const uint32_t *u, uint64_t count)
{
    uint64_t ones = 0;
    for (uint64_t i = 0; i < count; ++i) {
        uint32_t v = u[i];
        while (v) {
            ones += v & 1u;
            v >>= 1;
        }
    }
    return ones;
}

/* Frequency: histogram of the top 8 bits of every output (256 bins). */
void oracle_bat_bytes(const uint32_t *u, uint64_t count, uint64_t hist[256])
{
    memset(hist, 0, 256 * sizeof(uint64_t));
    for (uint64_t i = 0; i < count; ++i)
        hist[u[i] >> 24]++;
}

/* Serial: each stream's outputs taken in non-overlapping consecutive pairs
 * (u_{2k}, u_{2k+1}); the cell is the top 4 bits of the first and of the
 * second, 16 x 16 cells. */
void oracle_bat_serial(const uint32_t *u, uint64_t n_streams, uint64_t n_per_stream,
                       uint64_t hist[256])
{
    memset(hist, 0, 256 * sizeof(uint64_t));
    for (uint64_t s = 0; s < n_streams; ++s)
        for (uint64_t j = 0; j + 1 < n_per_stream; j += 2) {
            uint32_t a = u[j * n_streams + s] >> 28;
            uint32_t b = u[(j + 1) * n_streams + s] >> 28;
            hist[a * 16 + b]++;
        }
}

static int cmp_u32(const void *x, const void *y)
{
    uint32_t a = *(const uint32_t *)x, b = *(const uint32_t *)y;
    return a < b ? -1 : a > b;
}

/* Birthday spacings (Marsaglia): m = 512 birthdays in a year of 2^24 days,
 * the top 24 bits of 512 consecutive outputs of one stream.  Sort them; the
 * spacings are the first birthday and the differences of neighbours (m
 * values); sort the spacings; the statistic is the number of spacings equal
 * to the one before them.  Sample i is block i / n_streams (512 outputs) of
 * stream i % n_streams, for i below min(floor(n_per_stream / 512) *
 * n_streams, max_samples); hist[k] counts samples with k repeats, k < 15,
 * and hist[15] those with 15 or more.  Returns the number of samples. */
uint64_t oracle_bat_birthday(const uint32_t *u, uint64_t n_streams, uint64_t n_per_stream,
                             uint64_t max_samples, uint64_t hist[16])
{
    uint32_t b[512], d[512];
    uint64_t samples = 0;
    memset(hist, 0, 16 * sizeof(uint64_t));
    for (uint64_t blk = 0; (blk + 1) * 512 <= n_per_stream; ++blk)
        for (uint64_t s = 0; s < n_streams && samples < max_samples; ++s) {
            for (int i = 0; i < 512; ++i)
                b[i] = u[(blk * 512 + i) * n_streams + s] >> 8;
            qsort(b, 512, sizeof(uint32_t), cmp_u32);
            d[0] = b[0];
            for (int i = 1; i < 512; ++i)
                d[i] = b[i] - b[i - 1];
            qsort(d, 512, sizeof(uint32_t), cmp_u32);
            int repeats = 0;
            for (int i = 1; i < 512; ++i)
                repeats += d[i] == d[i - 1];
            hist[repeats < 15 ? repeats : 15]++;
            ++samples;
        }
    return samples;
}
