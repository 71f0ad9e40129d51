/* Bitsliced LFSRs and CRC-8 on GB300: the generic building blocks the paper
 * bitslices before MICKEY 2.0 (Sec. II-B and IV-C, Eq. 1 and 2: an n-bit
 * LFSR with feedback coefficients a_i; Sec. IV-B, Figs. CRC1 and CRC2: an
 * 8-bit CRC of 32 data streams at once).  Part of libmickey; the error
 * codes, memory kinds and MICKEY_API are those of mickey.h.
 *
 * One 32-bit word holds the same bit of 32 instances (lane l = instance
 * 32g + l of group g), so a clock of 32 LFSRs is a handful of full-width
 * logic ops, and the register shift is register renaming.
 */
#ifndef BITSLICE_LFSR_H
#define BITSLICE_LFSR_H

#include <stddef.h>
#include <stdint.h>

#include "mickey.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Fibonacci LFSRs (Eq. 1 and 2).  Instance i has an n-bit register
 * x_0 .. x_{n-1} (n = `degree`, 2..64) seeded with bit j of seeds[i] as x_j
 * (bits >= degree must be 0).  Each clock outputs x_0, computes
 * f = XOR over j of a_j x_j with a_j = bit j of `taps` (bits >= degree must
 * be 0, a_0 must be 1 so that the register is invertible), shifts
 * x_j <- x_{j+1} and sets x_{n-1} = f; the output sequence satisfies
 * s_{t+n} = XOR_j a_j s_{t+j}.
 *
 *   seeds   n_inst u64 (host or device per `mem`), read during the call.
 *   out     device pointer, word-major bitsliced: word (t, g) at
 *           out[t * G + g], G = ceil(n_inst / 32), bit l = output bit t of
 *           instance 32g + l (lanes past n_inst are 0); n_bits * G u32 words.
 *   stream  cudaStream_t (NULL: the default stream); asynchronous.
 * Returns 0, MICKEY_E_ARG (NULL pointer, n_inst or n_bits 0, degree outside
 * 2..64, taps outside the degree or a_0 = 0) or MICKEY_E_CUDA.
 * Up to 16 taps run in a kernel that reads only the taps' words (k - 1
 * XORs per clock), more in one that XORs all `degree` words under masks;
 * both give the same words.  Test hooks read at each call:
 * MICKEY_LFSR_DENSE=1 forces the mask kernel, MICKEY_LFSR_NOBATCH=1 makes
 * the few-tap kernel clock one step at a time. */
MICKEY_API int mickey_lfsr_generate(const uint64_t *seeds, size_t n_inst, int degree,
                                    uint64_t taps, uint64_t n_bits, uint32_t *out, int mem,
                                    void *stream);

/* CRC-8 (Sec. IV-B) of n messages of `len` bytes each, message i at
 * data + i * len (row-major).  Register preset `init`; every message bit,
 * bytes in order and each byte's most significant bit first, is XORed into
 * the register's top bit, the register moves up one place and takes the
 * polynomial's low 8 coefficients (bit k = coefficient of x^k; x^8 is
 * implicit) when that top bit was 1; the result is the register XOR
 * `xorout`.  crc[i] receives message i's CRC.
 *
 *   data, crc  host or device pointers per `mem` (both the same kind);
 *              data may be NULL when len is 0.
 *   stream     cudaStream_t; host memory makes the call synchronous.
 * Returns 0, MICKEY_E_ARG (NULL crc, or NULL data with len > 0) or
 * MICKEY_E_OOM / MICKEY_E_CUDA. */
MICKEY_API int mickey_crc8(const uint8_t *data, size_t n, size_t len, uint8_t poly,
                           uint8_t init, uint8_t xorout, uint8_t *crc, int mem, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BITSLICE_LFSR_H */
