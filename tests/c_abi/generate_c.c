/* A plain C user of the library: keys and IVs in, row-major keystream
 * bytes out, through include/mickey.h only (no CUDA headers, host memory).
 *
 *   generate_c <inputs> <n> <n_bits> <output>
 *
 * <inputs>: n * 10 key bytes followed by n * 10 IV bytes (80-bit IVs).
 * <output>: n rows of ceil(n_bits / 8) keystream bytes, MSB first.
 * Exit status 0 on success, else the library's error code (negated). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "mickey.h"

int main(int argc, char **argv) {
  if (argc != 5) {
    fprintf(stderr, "usage: %s inputs n n_bits output\n", argv[0]);
    return 2;
  }
  const size_t n = strtoull(argv[2], NULL, 10);
  const uint64_t n_bits = strtoull(argv[3], NULL, 10);
  uint8_t *in = malloc(20 * n);
  FILE *f = fopen(argv[1], "rb");
  if (!in || !f || fread(in, 1, 20 * n, f) != 20 * n) return 3;
  fclose(f);
  mickey_streams *s = mickey_init_streams(in, in + 10 * n, NULL, n);
  if (!s) {
    fprintf(stderr, "init: %s\n", mickey_last_error_message());
    return -mickey_last_error();
  }
  const size_t bytes = mickey_output_bytes(n, n_bits, MICKEY_LAYOUT_BYTES);
  uint8_t *out = malloc(bytes);
  int rc = out ? mickey_generate_host(s, n_bits, out, MICKEY_LAYOUT_BYTES) : MICKEY_E_OOM;
  if (rc == MICKEY_OK) rc = mickey_sync(s);
  if (rc != MICKEY_OK) {
    fprintf(stderr, "generate: %s\n", mickey_error_string(rc));
    mickey_free(s);
    return -rc;
  }
  f = fopen(argv[4], "wb");
  if (!f || fwrite(out, 1, bytes, f) != bytes) return 4;
  fclose(f);
  mickey_free(s);
  free(out);
  free(in);
  return 0;
}
