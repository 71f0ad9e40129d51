/* Scalar LFSR and CRC-8 oracle -- TEST INFRASTRUCTURE ONLY (see lfsr.py).
 *
 * Fibonacci LFSR of the paper's Sec. II-B / IV-C (Eq. 1 and 2): an n-bit
 * register x_0 .. x_{n-1} and feedback coefficients a_0 .. a_{n-1} in GF(2).
 * Each clock outputs x_0, computes the feedback bit f = XOR of a_i * x_i
 * over i, shifts every bit down one place (x_i <- x_{i+1}) and puts f in
 * x_{n-1}.  One bit per byte, one step per loop turn.
 *
 * CRC-8 of Sec. IV-B (Figs. CRC1/CRC2): an 8-bit register c_0 .. c_7 preset
 * to `init`; for each message bit m (bytes in order, each byte's most
 * significant bit first): f = c_7 XOR m, every bit moves up one place
 * (c_k <- c_{k-1}, c_0 <- 0), and if f = 1 the register is XORed with the
 * polynomial's low 8 coefficients (x^8 is implicit).  The result is the
 * register XOR `xorout`.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

int lfsr_oracle_generate(uint64_t seed, int degree, uint64_t taps, uint64_t n_bits,
                         uint8_t *bits) {
  if (degree < 2 || degree > 64) return -1;
  uint8_t x[64], a[64];
  for (int i = 0; i < degree; ++i) {
    x[i] = (uint8_t)((seed >> i) & 1u);
    a[i] = (uint8_t)((taps >> i) & 1u);
  }
  for (uint64_t t = 0; t < n_bits; ++t) {
    bits[t] = x[0];
    uint8_t f = 0;
    for (int i = 0; i < degree; ++i) f ^= (uint8_t)(a[i] & x[i]);
    for (int i = 0; i + 1 < degree; ++i) x[i] = x[i + 1];
    x[degree - 1] = f;
  }
  return 0;
}

uint8_t crc8_oracle(const uint8_t *msg, size_t len, uint8_t poly, uint8_t init,
                    uint8_t xorout) {
  uint8_t c[8], p[8];
  for (int k = 0; k < 8; ++k) {
    c[k] = (uint8_t)((init >> k) & 1u);
    p[k] = (uint8_t)((poly >> k) & 1u);
  }
  for (size_t j = 0; j < len; ++j) {
    for (int b = 7; b >= 0; --b) {
      const uint8_t m = (uint8_t)((msg[j] >> b) & 1u);
      const uint8_t f = (uint8_t)(c[7] ^ m);
      for (int k = 7; k > 0; --k) c[k] = c[k - 1];
      c[0] = 0;
      if (f)
        for (int k = 0; k < 8; ++k) c[k] ^= p[k];
    }
  }
  uint8_t r = 0;
  for (int k = 0; k < 8; ++k) r |= (uint8_t)(c[k] << k);
  return (uint8_t)(r ^ xorout);
}

typedef struct {
  const uint8_t *data;
  size_t len, lo, hi;
  uint8_t poly, init, xorout;
  uint8_t *out;
} crc_job;

static void *crc_worker(void *arg) {
  crc_job *j = (crc_job *)arg;
  for (size_t i = j->lo; i < j->hi; ++i)
    j->out[i] = crc8_oracle(j->data + i * j->len, j->len, j->poly, j->init, j->xorout);
  return NULL;
}

/* CRC of n messages of len bytes each (message i at data + i*len), on up
 * to `threads` threads (independent messages side by side). */
int crc8_oracle_batch(const uint8_t *data, size_t n, size_t len, uint8_t poly, uint8_t init,
                      uint8_t xorout, uint8_t *out, int threads) {
  if (threads < 1) threads = 1;
  if ((size_t)threads > n) threads = n ? (int)n : 1;
  pthread_t *tid = malloc(sizeof(pthread_t) * threads);
  crc_job *jobs = malloc(sizeof(crc_job) * threads);
  if (!tid || !jobs) {
    free(tid);
    free(jobs);
    return -1;
  }
  for (int t = 0; t < threads; ++t) {
    jobs[t] = (crc_job){data, len, n * t / threads, n * (t + 1) / threads, poly, init, xorout,
                        out};
    pthread_create(&tid[t], NULL, crc_worker, &jobs[t]);
  }
  for (int t = 0; t < threads; ++t) pthread_join(tid[t], NULL);
  free(tid);
  free(jobs);
  return 0;
}
