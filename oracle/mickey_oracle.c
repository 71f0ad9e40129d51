/*
 * Scalar MICKEY 2.0 oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, obviously-correct CPU statement of the
 * keystream generator whose bitsliced GPU form the library implements.
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or helper with the CUDA
 * path; it is built by plain gcc.
 *
 * What it computes
 * ----------------
 * MICKEY 2.0 (Babbage & Dodd), the stream cipher the paper bitslices
 * (Sec. II-C-1: two 100-bit registers R (linear) and S (non-linear), each
 * clocked irregularly under the control of the other; Sec. IV-D: the
 * bitsliced form keeps 200 words, one per register bit).  The paper does
 * not restate the cipher; the procedures below follow the designers'
 * specification that it cites, one function per procedure, each register
 * held as 100 separate bits (no packing, no word tricks):
 *
 *   CLOCK_R   linear register R with feedback taps RTAPS, optionally XORed
 *             with its own old value when its control bit is set;
 *   CLOCK_S   non-linear register S: intermediate value from COMP0/COMP1,
 *             then feedback through FB0 (control 0) or FB1 (control 1);
 *   CLOCK_KG  control bits CONTROL_BIT_R = s34^r67, CONTROL_BIT_S = s67^r33;
 *             in mixing mode the R input also takes s50; both registers
 *             are clocked from the old state;
 *   init      zero state, one mixing clock per IV bit, one per key bit
 *             (80), then 100 mixing clocks with input 0;
 *   keystream z = r0 ^ s0 taken before each non-mixing, zero-input clock.
 *
 * Readings where the paper is silent:
 *   - key bit k_i / IV bit iv_i is bit (7 - i%8) of byte i/8 (MSB first);
 *   - keystream bit z_t is written MSB-first: bit (7 - t%8) of byte t/8;
 *   - IV length is any integer 0..80 bits; the key is exactly 80 bits.
 *
 * Constant tables are kept as 100-character bit strings, index 0 first,
 * transcribed from the specification's tables.  RTAPS is the list of tap
 * positions of R.  COMP0/COMP1 are defined for i = 1..98 only; positions 0
 * and 99 hold '0' and are never read.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define MICKEY_REG 100

static const int RTAPS_LIST[] = {
    0,  1,  3,  4,  5,  6,  9,  12, 13, 16, 19, 20, 21, 22, 25, 28, 37,
    38, 41, 42, 45, 46, 50, 52, 54, 56, 58, 60, 61, 63, 64, 65, 66, 67,
    71, 72, 79, 80, 81, 82, 87, 88, 89, 90, 91, 92, 94, 95, 96, 97};

/* ten characters per chunk: indices 0-9, 10-19, ... */
static const char *COMP0_STR =
    "0000110001" "0111101001" "0101010101" "1010010000" "0001010101"
    "0000101001" "1110010101" "1111111101" "0111111010" "1000000110";
static const char *COMP1_STR =
    "0101100101" "1110010100" "0110101110" "1111000110" "1011100001"
    "0001011100" "0111111010" "1110111100" "0100001110" "0010011000";
static const char *FB0_STR =
    "1111010111" "1111100101" "1111111110" "0110000001" "1100100101"
    "0100101111" "0101010000" "0000011010" "0011011100" "1110011000";
static const char *FB1_STR =
    "1110111000" "0111010011" "0001001100" "1011000110" "0000110110"
    "0010001001" "0010110101" "0010100011" "1101111100" "0000100001";

typedef struct {
    uint8_t r[MICKEY_REG];
    uint8_t s[MICKEY_REG];
} mickey_oracle_state;

static uint8_t RTAPS[MICKEY_REG], COMP0[MICKEY_REG], COMP1[MICKEY_REG],
    FB0[MICKEY_REG], FB1[MICKEY_REG];
static pthread_once_t tables_once = PTHREAD_ONCE_INIT;

static void load_tables(void) {
    memset(RTAPS, 0, sizeof RTAPS);
    for (size_t k = 0; k < sizeof RTAPS_LIST / sizeof RTAPS_LIST[0]; ++k)
        RTAPS[RTAPS_LIST[k]] = 1;
    for (int i = 0; i < MICKEY_REG; ++i) {
        COMP0[i] = (uint8_t)(COMP0_STR[i] - '0');
        COMP1[i] = (uint8_t)(COMP1_STR[i] - '0');
        FB0[i] = (uint8_t)(FB0_STR[i] - '0');
        FB1[i] = (uint8_t)(FB1_STR[i] - '0');
    }
}
static void tables(void) { pthread_once(&tables_once, load_tables); }

/* Copy of the five tables, one byte (0/1) per position, for the tests. */
void mickey_oracle_tables(uint8_t *rtaps, uint8_t *comp0, uint8_t *comp1,
                          uint8_t *fb0, uint8_t *fb1) {
    tables();
    memcpy(rtaps, RTAPS, MICKEY_REG);
    memcpy(comp0, COMP0, MICKEY_REG);
    memcpy(comp1, COMP1, MICKEY_REG);
    memcpy(fb0, FB0, MICKEY_REG);
    memcpy(fb1, FB1, MICKEY_REG);
}

/* CLOCK_R: shift up by one, feedback r99^input into the tap positions,
 * and, when the control bit is set, XOR the old register in. */
void mickey_oracle_clock_r(mickey_oracle_state *st, int input_bit_r,
                           int control_bit_r) {
    tables();
    uint8_t old[MICKEY_REG], nr[MICKEY_REG];
    memcpy(old, st->r, MICKEY_REG);
    int feedback_bit = old[99] ^ (input_bit_r & 1);
    nr[0] = 0;
    for (int i = 1; i < MICKEY_REG; ++i) nr[i] = old[i - 1];
    if (feedback_bit)
        for (int i = 0; i < MICKEY_REG; ++i)
            if (RTAPS[i]) nr[i] ^= 1;
    if (control_bit_r & 1)
        for (int i = 0; i < MICKEY_REG; ++i) nr[i] ^= old[i];
    memcpy(st->r, nr, MICKEY_REG);
}

/* CLOCK_S: intermediate value s_hat from COMP0/COMP1, then the feedback
 * s99^input added through FB0 (control 0) or FB1 (control 1). */
void mickey_oracle_clock_s(mickey_oracle_state *st, int input_bit_s,
                           int control_bit_s) {
    tables();
    uint8_t old[MICKEY_REG], hat[MICKEY_REG];
    memcpy(old, st->s, MICKEY_REG);
    int feedback_bit = old[99] ^ (input_bit_s & 1);
    hat[0] = 0;
    for (int i = 1; i <= 98; ++i)
        hat[i] = old[i - 1] ^ ((old[i] ^ COMP0[i]) & (old[i + 1] ^ COMP1[i]));
    hat[99] = old[98];
    const uint8_t *fb = (control_bit_s & 1) ? FB1 : FB0;
    for (int i = 0; i < MICKEY_REG; ++i)
        st->s[i] = hat[i] ^ (fb[i] & feedback_bit);
}

/* CLOCK_KG: both control bits and the R input come from the old state. */
void mickey_oracle_clock_kg(mickey_oracle_state *st, int mixing,
                            int input_bit) {
    int control_bit_r = st->s[34] ^ st->r[67];
    int control_bit_s = st->s[67] ^ st->r[33];
    int input_bit_r = (input_bit & 1) ^ (mixing ? st->s[50] : 0);
    int input_bit_s = input_bit & 1;
    mickey_oracle_clock_r(st, input_bit_r, control_bit_r);
    mickey_oracle_clock_s(st, input_bit_s, control_bit_s);
}

static int get_bit_msb_first(const uint8_t *bytes, uint32_t i) {
    return (bytes[i >> 3] >> (7 - (i & 7))) & 1;
}

/* Key/IV loading: zero state, IV bits, 80 key bits, 100 preclocks, all in
 * mixing mode.  iv may be NULL when iv_len == 0.  Returns 0, or -1 when
 * iv_len exceeds 80 bits. */
int mickey_oracle_init(mickey_oracle_state *st, const uint8_t *key,
                       const uint8_t *iv, uint32_t iv_len) {
    if (iv_len > 80) return -1;
    memset(st, 0, sizeof *st);
    for (uint32_t i = 0; i < iv_len; ++i)
        mickey_oracle_clock_kg(st, 1, get_bit_msb_first(iv, i));
    for (uint32_t i = 0; i < 80; ++i)
        mickey_oracle_clock_kg(st, 1, get_bit_msb_first(key, i));
    for (int i = 0; i < 100; ++i) mickey_oracle_clock_kg(st, 1, 0);
    return 0;
}

/* Keystream: for each bit, z = r0 ^ s0, then one non-mixing zero-input
 * clock.  Bits are OR-ed into out (MSB first) starting at bit offset
 * `bit_offset`; the caller zeroes out beforehand. */
void mickey_oracle_keystream(mickey_oracle_state *st, uint64_t n_bits,
                             uint8_t *out, uint64_t bit_offset) {
    for (uint64_t t = 0; t < n_bits; ++t) {
        int z = st->r[0] ^ st->s[0];
        uint64_t b = bit_offset + t;
        if (z) out[b >> 3] |= (uint8_t)(0x80u >> (b & 7));
        mickey_oracle_clock_kg(st, 0, 0);
    }
}

/* One stream end to end: init then n_bits of keystream into out
 * (ceil(n_bits/8) bytes, zero-padded).  Returns 0 or -1 (bad iv_len). */
int mickey_oracle_stream(const uint8_t *key, const uint8_t *iv,
                         uint32_t iv_len, uint64_t n_bits, uint8_t *out) {
    mickey_oracle_state st;
    if (mickey_oracle_init(&st, key, iv, iv_len)) return -1;
    memset(out, 0, (size_t)((n_bits + 7) / 8));
    mickey_oracle_keystream(&st, n_bits, out, 0);
    return 0;
}

/* ---- many independent streams over host threads (one stream per task) --- */

typedef struct {
    size_t n;
    const uint8_t *keys, *ivs;          /* n x 10 bytes each */
    const uint32_t *iv_lens;            /* n values */
    const uint64_t *n_bits;             /* n values */
    uint8_t *out;                       /* bytes, stream i at out_offsets[i] */
    const uint64_t *out_offsets;
    size_t next;
    int status;
    pthread_mutex_t lock;
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *job = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        size_t i = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (i >= job->n) break;
        if (mickey_oracle_stream(job->keys + 10 * i, job->ivs + 10 * i,
                                 job->iv_lens[i], job->n_bits[i],
                                 job->out + job->out_offsets[i])) {
            pthread_mutex_lock(&job->lock);
            job->status = -1;
            pthread_mutex_unlock(&job->lock);
        }
    }
    return NULL;
}

/* Runs n streams on `threads` host threads (<= 0 means 1).  Stream i writes
 * ceil(n_bits[i]/8) bytes at out + out_offsets[i].  Returns 0, or -1 if some
 * iv_len exceeded 80 or a thread could not be started. */
int mickey_oracle_batch(size_t n, const uint8_t *keys, const uint8_t *ivs,
                        const uint32_t *iv_lens, const uint64_t *n_bits,
                        uint8_t *out, const uint64_t *out_offsets,
                        int threads) {
    tables();
    batch_job job = {n, keys, ivs, iv_lens, n_bits, out, out_offsets, 0, 0,
                     PTHREAD_MUTEX_INITIALIZER};
    if (threads <= 1) {
        batch_worker(&job);
        return job.status;
    }
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!tid) return -1;
    int started = 0;
    for (int k = 0; k < threads; ++k) {
        if (pthread_create(&tid[k], NULL, batch_worker, &job)) break;
        ++started;
    }
    if (started == 0) batch_worker(&job);
    for (int k = 0; k < started; ++k) pthread_join(tid[k], NULL);
    free(tid);
    return job.status;
}

size_t mickey_oracle_state_size(void) { return sizeof(mickey_oracle_state); }
