/*
 * grain.h -- C ABI of the bitsliced Grain keystream generator (GB300,
 * sm_103a), the paper's second stream cipher (Sec. II-C-3: an 80-bit LFSR
 * and an 80-bit NFSR shifted together each clock, an 80-bit key loaded into
 * the NFSR and a 64-bit IV into the LFSR, 160 initialisation clocks with
 * the output fed back, then one keystream bit per clock).  Bitsliced as in
 * Sec. IV-A/IV-D: a 32-bit word holds the same register bit of 32
 * instances; instances 32g .. 32g+31 form group g.
 *
 * Conventions (the specification's test vectors fix the bit order):
 *  keys     n x 10 bytes; key bit i is bit (i % 8) of byte i/8.
 *  ivs      n x 8 bytes; IV bit i is bit (i % 8) of byte i/8.
 *  output   MICKEY_LAYOUT_BITSLICED_U32: uint32 [G][n_bits], word [g][t]
 *           bit l = z_t of instance 32g + l, lanes past n - 1 zero;
 *           MICKEY_LAYOUT_BYTES: uint8 [n][ceil(n_bits / 8)], keystream bit
 *           t of a call at bit (t % 8) of byte t/8 (least significant first),
 *           unused high bits of a last partial byte zero.
 *  Errors   as in mickey.h: MICKEY_OK or a negative MICKEY_E_* code, the
 *           cause in mickey_last_error() / mickey_last_error_message().
 *  Streams  work is enqueued on the handle's CUDA stream; calls return once
 *           it is enqueued.
 *  Launch   with no more 32-group warp-groups than resident warps, one warp
 *           per warp-group clocks the whole call; with more, a persistent
 *           launch takes (warp-group, 1280-clock chunk) items from a queue,
 *           each chunk continuing from the state its predecessor published
 *           (a bounded wait: MICKEY_SPIN_LIMIT polls of about 256 ns, after
 *           which grain_sync reports MICKEY_E_TIMEOUT).  MICKEY_GRAIN_QUEUE=1,
 *           read when a handle is created, forces the queue.  The bytes
 *           layout stages rows in tensor memory (one block of 8 warps per SM).
 */
#ifndef GRAIN_H
#define GRAIN_H

#include <stddef.h>
#include <stdint.h>

#include "mickey.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grain_streams grain_streams;

/* n instances: key/IV loading and the 160 initialisation clocks (Sec.
 * II-C-3), bitsliced on the device.  keys/ivs in `mem` (MICKEY_MEM_HOST:
 * copied; MICKEY_MEM_DEVICE: must stay valid until the work is done).
 * NULL on error (MICKEY_E_ARG, MICKEY_E_OOM, MICKEY_E_CUDA). */
MICKEY_API grain_streams *grain_init_streams(const void *keys, const void *ivs, size_t n, int mem,
                                             void *cuda_stream);

/* Re-key the handle in place (same n, no device allocation after the
 * first call with host inputs): loading and the 160 initialisation clocks
 * again; the position returns to 0. */
MICKEY_API int grain_reset_streams(grain_streams *s, const void *keys, const void *ivs, int mem);

/* The next n_bits keystream bits of every instance (1 .. 2^34 per call) into
 * the caller-owned DEVICE buffer `out` (grain_output_bytes bytes).  Stateful:
 * each call continues every stream.  Errors: MICKEY_E_ARG, MICKEY_E_LAYOUT
 * (a layout other than the two above), MICKEY_E_CUDA. */
MICKEY_API int grain_generate(grain_streams *s, uint64_t n_bits, void *out, int layout);
MICKEY_API size_t grain_output_bytes(size_t n, uint64_t n_bits, int layout);

MICKEY_API int grain_set_stream(grain_streams *s, void *cuda_stream);
/* Wait for the handle's stream; MICKEY_E_TIMEOUT if a queue wait ran out. */
MICKEY_API int grain_sync(grain_streams *s);
/* Keystream bits generated so far (the same for every instance). */
MICKEY_API uint64_t grain_position(const grain_streams *s);
/* Every instance's state, 20 bytes: LFSR bits s0..s79 in bytes 0..9, NFSR
 * bits b0..b79 in bytes 10..19, bit k at bit (k % 8) of byte k/8 of the
 * record (synchronises). */
MICKEY_API int grain_export_state(grain_streams *s, uint8_t *states);
/* Logic operations of one bitsliced clock of a 32-lane group (init != 0:
 * an initialisation clock), as the kernels compute it.  Host-only. */
MICKEY_API int grain_ops_per_clock(int init);
MICKEY_API void grain_free(grain_streams *s);

/* Measurement helper: the bare bitsliced Grain clock (blocks_per_sm 1..4
 * blocks of 64 threads per SM, one 32-lane group per thread, bodies x 80
 * clocks from an arbitrary state; store != 0 also writes each clock's
 * keystream word to shared memory), synchronously on the current device.
 * Outputs (each may be NULL): grain_ops_per_clock(0) ops per group-clock per
 * SM per SM-cycle, and the SM clock seen (MHz) -- the ceiling of the
 * keystream kernels' clock at that many warps per SM. */
MICKEY_API int grain_probe_clock(int blocks_per_sm, int bodies, int store, double *ops_per_sm_clk,
                                 double *sm_mhz);

#ifdef __cplusplus
}
#endif

#endif /* GRAIN_H */
