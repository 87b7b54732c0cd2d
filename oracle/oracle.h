/*
 * Oracle for Hissoiny, Despres & Ozell, "Using graphics processing units to
 * generate random numbers" (arXiv:1101.1846): plain single-threaded C.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline / reference arm may.  It shares no source, header, table or helper
 * with the CUDA library under paper_1101_1846_gb300/csrc/.
 *
 * Generator kinds and output formats (numbering shared with the C-ABI only
 * as plain integers, so that the two sides can be called with the same
 * arguments):
 *   kind 0 = multiply-with-carry, base 2^32            (Eq. 2-3)
 *   kind 1 = xor128 XorShift, 4 x 32-bit words          (Marsaglia 2003, the
 *            paper's reference for XorShift generators)
 *   kind 2 = KISS = MWC + xorshift32 + LCG mod 2^32     (Eq. 6, Eq. 7 and the
 *            KISS section; sum form)
 *   kind 3 = the paper's own MWC: two base-2^16 MWCs joined as (z << 16) + w
 *            (Methods / MWC)
 *   kind 4 = Panneton's XorShift, r = 8 words, s = 7 (Eq. 5)
 *   kind 5 = KISS in the paper's form ((MWC xor LCG) + xorshift32, with the
 *            kind-3 MWC; Background / KISS)
 *   fmt 0 = uint32, fmt 1 = float32 uniform (u >> 8) * 2^-24
 *
 * Per-stream state: oracle_state_words(kind) 32-bit words (8 for kind 4,
 * else 4), st[0..]:
 *   MWC       {x, c, 0, 0}
 *   xor128    {x, y, z, w}
 *   KISS      {x, c, y, z}  (MWC x and carry c, xorshift32 y, LCG z)
 *   MWC16X2   {z, w, 0, 0}  (each x | c << 16)
 *   XORSHIFT8 {v_{n-8}, ..., v_{n-1}}
 *   KISS_XOR  {z, w, y, z_lcg}
 * Kinds 3 and 5 take one packed multiplier pair a1 | a2 << 16 per stream.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* number theory */
uint64_t oracle_mulmod_u64(uint64_t a, uint64_t b, uint64_t m);
uint64_t oracle_powmod_u64(uint64_t base, uint64_t e, uint64_t m);
int oracle_is_prime_u64(uint64_t n);
int oracle_is_safe_multiplier(uint64_t a, int log2b);
uint64_t oracle_multipliers(int log2b, uint64_t a_top, uint64_t k, uint32_t *out);
uint64_t oracle_multipliers_range(int log2b, uint64_t a_hi, uint64_t a_lo,
                                  uint32_t *out, uint64_t cap);
uint64_t oracle_mwc16_pairs(uint64_t k, uint32_t *out);

/* seeding */
uint64_t oracle_splitmix64(uint64_t *z);
void oracle_seed_stream(int kind, uint32_t a, uint64_t seed, uint64_t s,
                        uint32_t *st);
void oracle_seed_streams(int kind, const uint32_t *a, uint64_t seed,
                         const uint64_t *s_ids, uint64_t n, uint32_t *st);

/* single steps */
uint32_t oracle_mwc_step(uint32_t a, uint32_t *x, uint32_t *c, int log2b);
uint32_t oracle_xor128_step(uint32_t st[4]);
uint32_t oracle_xorshift32_step(uint32_t *y);
uint32_t oracle_lcg_step(uint32_t *z);
uint32_t oracle_kiss_step(uint32_t a, uint32_t st[4]);
uint32_t oracle_mwc16x2_step(uint32_t a_pair, uint32_t st[2]);
uint32_t oracle_xorshift8_step(uint32_t st[8]);
uint32_t oracle_kiss_xor_step(uint32_t a_pair, uint32_t st[4]);
uint32_t oracle_step(int kind, uint32_t a, uint32_t *st);
int oracle_state_words(int kind);
float oracle_to_unit_f32(uint32_t u);

/* whole calls */
void oracle_stream(int kind, uint32_t a, uint32_t *st, uint64_t n, int fmt,
                   void *out);
void oracle_generate(int kind, uint64_t n_streams, const uint32_t *a,
                     uint32_t *state, uint64_t n_per_stream, int fmt,
                     void *out);

/* consumers with no output array (Sec. "Performance evaluation": numbers
 * used inline, only the final state stored) */
uint64_t oracle_sum_u32(const uint32_t *u, uint64_t n);
uint64_t oracle_sum_u24(const uint32_t *u, uint64_t n);
uint64_t oracle_disc_count(const uint32_t *u, uint64_t n);
int oracle_reduce(int kind, uint64_t n_streams, const uint32_t *a,
                  uint32_t *state, uint64_t n_per_stream, int op,
                  uint64_t *out);

/* jump-ahead by k steps (Sec. "Parallelizing RNGs", sequence splitting) */
void oracle_mwc_jump(uint32_t a, uint32_t *x, uint32_t *c, uint64_t k,
                     int log2b);
void oracle_xor128_jump(uint32_t st[4], uint64_t k);
void oracle_xorshift32_jump(uint32_t *y, uint64_t k);
void oracle_xorshift8_jump(uint32_t st[8], uint64_t k);
void oracle_lcg_jump(uint32_t *z, uint64_t k);
void oracle_jump(int kind, uint32_t a, uint32_t *st, uint64_t k);

/* statistical battery counts over stream-interleaved outputs (the paper's
 * randomness assessment, Sec. "Performance evaluation") */
uint64_t oracle_bat_ones(const uint32_t *u, uint64_t count);
void oracle_bat_bytes(const uint32_t *u, uint64_t count, uint64_t hist[256]);
void oracle_bat_serial(const uint32_t *u, uint64_t n_streams, uint64_t n_per_stream,
                       uint64_t hist[256]);
#define ORACLE_BAT_BIRTHDAY_MAX ((uint64_t)1 << 21)
uint64_t oracle_bat_birthday(const uint32_t *u, uint64_t n_streams, uint64_t n_per_stream,
                             uint64_t max_samples, uint64_t hist[16]);

/* brute-force periods (pins) */
uint64_t oracle_mwc_period(uint32_t a, uint32_t x0, uint32_t c0, int log2b,
                           uint64_t limit);
uint64_t oracle_xorshift32_period(uint32_t y0);
uint64_t oracle_lcg_period(uint32_t z0);

#ifdef __cplusplus
}
#endif
#endif
