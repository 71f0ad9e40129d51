/*
 * Scalar Grain oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously-correct CPU statement of the
 * keystream generator whose bitsliced GPU form the library implements for
 * the paper's second stream cipher (Sec. II-C-3: Grain, Hell et al., two
 * 80-bit shift registers, an LFSR and an NFSR, shifted together each clock;
 * 80-bit key into the NFSR, 64-bit IV into the LFSR; 160 initialisation
 * clocks before the keystream).  Only the test-suite and the benchmark's
 * CPU leg may load it.  It shares no code, header or table with the CUDA
 * path; it is built by plain gcc.
 *
 * What it computes (Grain v1, the eSTREAM portfolio version the paper's
 * citation describes), each register held as 80 separate bits s[0..79]
 * (LFSR) and b[0..79] (NFSR), s[0] / b[0] the oldest:
 *
 *   LFSR feedback   s_{i+80} = s_{i+62} + s_{i+51} + s_{i+38} + s_{i+23}
 *                              + s_{i+13} + s_i
 *   NFSR feedback   b_{i+80} = s_i + g(b), with g the specification's
 *                   non-linear function of b_i .. b_{i+63} (linear terms of
 *                   11 taps plus 11 products of 2 to 6 taps)
 *   filter          h(x0..x4) = x1 + x4 + x0x3 + x2x3 + x3x4 + x0x1x2
 *                   + x0x2x3 + x0x2x4 + x1x2x4 + x2x3x4 of
 *                   (s_{i+3}, s_{i+25}, s_{i+46}, s_{i+64}, b_{i+63})
 *   output          z_i = sum of b_{i+k}, k in {1, 2, 4, 10, 31, 43, 56},
 *                   + h(...)
 *   initialisation  b_i = key bit i, s_i = IV bit i (i < 64), s_i = 1
 *                   (64 <= i < 80); 160 clocks in which the output z is
 *                   not emitted but added into both feedbacks.
 *
 * Bit order (fixed by the specification's test vectors, which this order
 * reproduces): key/IV bit i is bit (i % 8) of byte i/8 (least significant
 * first); keystream bit t is written to bit (t % 8) of byte t/8.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GRAIN_REG 80

typedef struct {
    uint8_t s[GRAIN_REG]; /* LFSR */
    uint8_t b[GRAIN_REG]; /* NFSR */
} grain_oracle_state;

static uint8_t lfsr_feedback(const uint8_t *s) {
    return s[62] ^ s[51] ^ s[38] ^ s[23] ^ s[13] ^ s[0];
}

/* g(b): the non-linear part of the NFSR feedback (without the s_i term). */
static uint8_t nfsr_g(const uint8_t *b) {
    uint8_t v = b[62] ^ b[60] ^ b[52] ^ b[45] ^ b[37] ^ b[33] ^ b[28] ^ b[21] ^ b[14] ^ b[9] ^
                b[0];
    v ^= b[63] & b[60];
    v ^= b[37] & b[33];
    v ^= b[15] & b[9];
    v ^= b[60] & b[52] & b[45];
    v ^= b[33] & b[28] & b[21];
    v ^= b[63] & b[45] & b[28] & b[9];
    v ^= b[60] & b[52] & b[37] & b[33];
    v ^= b[63] & b[60] & b[21] & b[15];
    v ^= b[63] & b[60] & b[52] & b[45] & b[37];
    v ^= b[33] & b[28] & b[21] & b[15] & b[9];
    v ^= b[52] & b[45] & b[37] & b[33] & b[28] & b[21];
    return v;
}

static uint8_t filter_h(uint8_t x0, uint8_t x1, uint8_t x2, uint8_t x3, uint8_t x4) {
    return x1 ^ x4 ^ (x0 & x3) ^ (x2 & x3) ^ (x3 & x4) ^ (x0 & x1 & x2) ^ (x0 & x2 & x3) ^
           (x0 & x2 & x4) ^ (x1 & x2 & x4) ^ (x2 & x3 & x4);
}

/* z_i of the current state. */
uint8_t grain_oracle_output(const grain_oracle_state *st) {
    const uint8_t *s = st->s, *b = st->b;
    uint8_t z = b[1] ^ b[2] ^ b[4] ^ b[10] ^ b[31] ^ b[43] ^ b[56];
    return z ^ filter_h(s[3], s[25], s[46], s[64], b[63]);
}

/* One clock of both registers; `extra` is added into both new bits (the
 * output during initialisation, 0 afterwards). */
void grain_oracle_clock(grain_oracle_state *st, int extra) {
    const uint8_t ns = lfsr_feedback(st->s) ^ (uint8_t)(extra & 1);
    const uint8_t nb = st->s[0] ^ nfsr_g(st->b) ^ (uint8_t)(extra & 1);
    memmove(st->s, st->s + 1, GRAIN_REG - 1);
    memmove(st->b, st->b + 1, GRAIN_REG - 1);
    st->s[GRAIN_REG - 1] = ns;
    st->b[GRAIN_REG - 1] = nb;
}

static int bit_lsb_first(const uint8_t *bytes, int i) { return (bytes[i / 8] >> (i % 8)) & 1; }

/* key: 10 bytes, iv: 8 bytes. */
void grain_oracle_init(grain_oracle_state *st, const uint8_t *key, const uint8_t *iv) {
    for (int i = 0; i < GRAIN_REG; ++i) st->b[i] = (uint8_t)bit_lsb_first(key, i);
    for (int i = 0; i < 64; ++i) st->s[i] = (uint8_t)bit_lsb_first(iv, i);
    for (int i = 64; i < GRAIN_REG; ++i) st->s[i] = 1;
    for (int t = 0; t < 160; ++t) grain_oracle_clock(st, grain_oracle_output(st));
}

/* n_bits keystream bits OR-ed into out (bit t at bit t%8 of byte t/8, t
 * counted from bit_offset), continuing the state. */
void grain_oracle_keystream(grain_oracle_state *st, uint64_t n_bits, uint8_t *out,
                            uint64_t bit_offset) {
    for (uint64_t t = 0; t < n_bits; ++t) {
        const uint64_t k = t + bit_offset;
        out[k / 8] |= (uint8_t)(grain_oracle_output(st) << (k % 8));
        grain_oracle_clock(st, 0);
    }
}

void grain_oracle_stream(const uint8_t *key, const uint8_t *iv, uint64_t n_bits, uint8_t *out) {
    grain_oracle_state st;
    grain_oracle_init(&st, key, iv);
    memset(out, 0, (size_t)((n_bits + 7) / 8));
    grain_oracle_keystream(&st, n_bits, out, 0);
}

/* ---- many independent streams over host threads (one stream per task) --- */

typedef struct {
    size_t n;
    const uint8_t *keys, *ivs; /* n x 10 and n x 8 bytes */
    uint64_t n_bits;
    uint8_t *out; /* n x ceil(n_bits/8) bytes */
    size_t next;
    pthread_mutex_t lock;
} grain_job;

static void *grain_worker(void *arg) {
    grain_job *job = (grain_job *)arg;
    const size_t row = (size_t)((job->n_bits + 7) / 8);
    for (;;) {
        pthread_mutex_lock(&job->lock);
        size_t i = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (i >= job->n) break;
        grain_oracle_stream(job->keys + 10 * i, job->ivs + 8 * i, job->n_bits, job->out + row * i);
    }
    return NULL;
}

/* n streams of n_bits each on `threads` host threads (<= 1 means one);
 * returns 0, or -1 if no thread could be started. */
int grain_oracle_batch(size_t n, const uint8_t *keys, const uint8_t *ivs, uint64_t n_bits,
                       uint8_t *out, int threads) {
    grain_job job = {n, keys, ivs, n_bits, out, 0, PTHREAD_MUTEX_INITIALIZER};
    if (threads <= 1) {
        grain_worker(&job);
        return 0;
    }
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!tid) return -1;
    int started = 0;
    for (int k = 0; k < threads; ++k) {
        if (pthread_create(&tid[k], NULL, grain_worker, &job)) break;
        ++started;
    }
    if (started == 0) grain_worker(&job);
    for (int k = 0; k < started; ++k) pthread_join(tid[k], NULL);
    free(tid);
    return 0;
}

size_t grain_oracle_state_size(void) { return sizeof(grain_oracle_state); }
