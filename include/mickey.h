/*
 * mickey.h -- C ABI of the bitsliced MICKEY 2.0 keystream library for GB300
 * (sm_103a).
 *
 * The library generates MICKEY 2.0 keystreams for many independent
 * (key, IV) instances at once.  Internally it uses the column-major
 * "bitsliced" representation of Sec. IV-A: a 32-bit word holds the same
 * register bit of 32 instances, so one GPU thread clocks 32 ciphers
 * (Sec. IV-D: 200 words for the 100-bit R and S registers).  Instances
 * 32g .. 32g+31 form group g.
 *
 * Conventions used by every entry point
 * -------------------------------------
 *  keys      n x 10 bytes, instance-major.  Key bit k_i is bit (7 - i%8) of
 *            byte i/8 (MSB first).
 *  ivs       n x 10 bytes.  Only the first iv_lens[i] bits of row i are
 *            used, same bit order.
 *  iv_lens   n values in [0, 80]; NULL means 80 for every instance.
 *  keystream bit z_t of an instance is the t-th output bit after the
 *            key/IV loading and the 100 preclocks of the cipher.
 *  Errors    functions returning int give MICKEY_OK (0) or a negative
 *            MICKEY_E_* code; functions returning a pointer give NULL.  In
 *            both cases mickey_last_error() and mickey_last_error_message()
 *            report the cause (thread-local).  Errors raised inside a kernel
 *            surface at the next mickey_sync() on that handle.
 *  Streams   device work is enqueued on the CUDA stream given at creation
 *            or by mickey_set_stream() (a cudaStream_t passed as void*;
 *            NULL is the legacy default stream).  Calls return once the
 *            work is enqueued unless stated otherwise.
 *  Threads   a handle must not be used by two host threads at once.
 *
 * Output layouts (argument `layout`), for a call producing n_bits per
 * instance:
 *  MICKEY_LAYOUT_BITSLICED_U32 (0)  uint32 [G][n_bits], G = ceil(n/32):
 *        word [g][t] has bit l = z_t of instance 32g+l (Sec. IV-A layout);
 *        bits of lanes past instance n-1 are zero.  Size 4*G*n_bits bytes.
 *  MICKEY_LAYOUT_BYTES (1)  uint8 [n][ceil(n_bits/8)], row-major: byte j of
 *        row i holds z_{8j..8j+7} of instance i, z_{8j} in bit 7; unused low
 *        bits of a last partial byte are zero.
 *  MICKEY_LAYOUT_U32 (2)  uint32 [n][n_bits/32]: word k of row i holds
 *        z_{32k..32k+31}, z_{32k} in bit 31.  Needs n_bits % 32 == 0.
 *  MICKEY_LAYOUT_U32_F32 (3)  the U32 array followed by float32
 *        [n][n_bits/32] with f = (w >> 8) * 2^-24 for the same word w: an
 *        exact uniform on [0, 1 - 2^-24].  Needs n_bits % 32 == 0.
 */
#ifndef MICKEY_H
#define MICKEY_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MICKEY_API __attribute__((visibility("default")))
#else
#define MICKEY_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define MICKEY_OK 0
#define MICKEY_E_ARG (-1)     /* NULL pointer, zero/oversized count, bad flag */
#define MICKEY_E_IVLEN (-2)   /* an IV length above 80 bits */
#define MICKEY_E_LIMIT (-3)   /* more than 2^40 keystream bits per key/IV */
#define MICKEY_E_LAYOUT (-4)  /* unknown layout or n_bits it cannot hold */
#define MICKEY_E_OOM (-5)     /* device or host allocation failed */
#define MICKEY_E_CUDA (-6)    /* a CUDA runtime call failed */
#define MICKEY_E_TIMEOUT (-7) /* a bounded device-side wait ran out */
#define MICKEY_E_STATE (-8)   /* handle not usable for this call */

#define MICKEY_LAYOUT_BITSLICED_U32 0
#define MICKEY_LAYOUT_BYTES 1
#define MICKEY_LAYOUT_U32 2
#define MICKEY_LAYOUT_U32_F32 3

#define MICKEY_MEM_HOST 0   /* pointer arguments are host memory */
#define MICKEY_MEM_DEVICE 1 /* pointer arguments are device memory */

#define MICKEY_KEY_BYTES 10
#define MICKEY_MAX_IV_BITS 80
/* Sec. II-C-1: up to 2^40 keystream bits may be produced per key/IV pair. */
#define MICKEY_MAX_STREAM_BITS (1ull << 40)

typedef struct mickey_streams mickey_streams;

/* --------------------------------------------------------------------------
 * Creation: key/IV loading and preclocking (Sec. IV-D; the cipher's
 * initialisation of the specification the paper cites): R = S = 0, one
 * mixing clock per IV bit, one per key bit, then 100 mixing clocks with
 * input 0 -- for all n instances, bitsliced, on the device.
 * ------------------------------------------------------------------------ */

/* Host inputs, legacy default stream.  The library copies keys, ivs and
 * iv_lens; the caller keeps ownership.  Errors: MICKEY_E_ARG (keys or ivs
 * NULL, n == 0), MICKEY_E_IVLEN, MICKEY_E_OOM, MICKEY_E_CUDA. */
MICKEY_API mickey_streams *mickey_init_streams(const uint8_t *keys, const uint8_t *ivs,
                                    const uint32_t *iv_lens, size_t n);

/* As mickey_init_streams, with the inputs' memory space `mem`
 * (MICKEY_MEM_HOST or MICKEY_MEM_DEVICE) and the CUDA stream the handle
 * uses from now on.  Device inputs must stay valid until the work is done
 * (mickey_sync); an IV length above 80 in device memory is reported as
 * MICKEY_E_IVLEN by mickey_sync. */
MICKEY_API mickey_streams *mickey_init_streams_ex(const void *keys, const void *ivs,
                                       const uint32_t *iv_lens, size_t n,
                                       int mem, void *cuda_stream);

/* Re-key an existing handle in place (same n, no allocation): runs the
 * whole loading and preclocking again and resets every position to 0. */
MICKEY_API int mickey_reset_streams(mickey_streams *s, const void *keys, const void *ivs,
                         const uint32_t *iv_lens, int mem);

/* Use `cuda_stream` for this handle's later work. */
MICKEY_API int mickey_set_stream(mickey_streams *s, void *cuda_stream);

/* --------------------------------------------------------------------------
 * Keystream: for t in 0..n_bits-1, z_t = r0 ^ s0, then one non-mixing
 * CLOCK_KG with input 0, for every instance (Sec. IV-D: 32 keystream bits per
 * thread per clock).  Stateful: each call continues every stream where the
 * previous call stopped.  `out` is a caller-owned DEVICE buffer of
 * mickey_output_bytes(n, n_bits, layout) bytes.
 * Errors: MICKEY_E_ARG (s or out NULL, n_bits == 0 or above 2^34 per call,
 * out not 4-byte aligned for a 32-bit layout), MICKEY_E_LAYOUT,
 * MICKEY_E_LIMIT (a stream would pass 2^40 bits), MICKEY_E_CUDA.
 * ------------------------------------------------------------------------ */
MICKEY_API int mickey_generate(mickey_streams *s, uint64_t n_bits, void *out, int layout);

/* Bytes one call writes for n instances and n_bits per instance; 0 when the
 * layout cannot hold n_bits. */
MICKEY_API size_t mickey_output_bytes(size_t n, uint64_t n_bits, int layout);

/* --------------------------------------------------------------------------
 * Ragged keystream (Sec. IV-D's one-instance-per-lane design with uneven
 * lengths): stream i continues by its own n_bits[i] bits (0 allowed, at most
 * 2^34 per call), in one launch.  Each 32-lane group is clocked as often as
 * its longest lane; every stream's state and position afterwards are those
 * after exactly its own n_bits[i] bits, so a later call (ragged or
 * mickey_generate) continues each stream exactly.
 *
 *  n_bits       host array of n values (n = mickey_num_streams); copied.
 *  out          caller-owned DEVICE buffer; nothing is written outside the
 *               rows and arrays described below.
 *  out_offsets  host array of byte offsets into out (copied), or NULL for
 *               the packed arrangement: rows (or group arrays) back to back
 *               in stream (group) order, mickey_ragged_output_bytes bytes.
 *  layout       MICKEY_LAYOUT_BYTES: stream i's ceil(n_bits[i] / 8) bytes at
 *                 out + out_offsets[i], as one row of the bytes layout (any
 *                 alignment);
 *               MICKEY_LAYOUT_U32: stream i's n_bits[i] / 32 words at
 *                 out + out_offsets[i] (4-byte aligned; n_bits[i] % 32 == 0);
 *               MICKEY_LAYOUT_BITSLICED_U32: out_offsets has ceil(n / 32)
 *                 entries; group g's C_g words at out + out_offsets[g]
 *                 (4-byte aligned; 16 for vector stores), C_g the longest
 *                 n_bits of its lanes; bit l of word t is z_t of instance
 *                 32g + l while t < n_bits[32g + l], else 0.
 * Equal lengths at the packed offsets are mickey_generate's layout and run
 * as its keystream launch.
 * Asynchronous on the handle's stream.  Errors (nothing is launched and no
 * position moves): MICKEY_E_ARG (NULL pointer, a length above 2^34, a
 * misaligned 32-bit output), MICKEY_E_LAYOUT (MICKEY_LAYOUT_U32_F32, or a
 * u32 length not a multiple of 32), MICKEY_E_LIMIT (a stream would pass 2^40
 * bits), MICKEY_E_OOM / MICKEY_E_CUDA.
 * ------------------------------------------------------------------------ */
MICKEY_API int mickey_generate_ragged(mickey_streams *s, const uint64_t *n_bits, void *out,
                                      const uint64_t *out_offsets, int layout);

/* Size in bytes of the packed output of mickey_generate_ragged for these n
 * lengths; 0 for a layout it does not take, a u32 length not a multiple of
 * 32, or a length above 2^34 (the per-call limit). */
MICKEY_API size_t mickey_ragged_output_bytes(size_t n, const uint64_t *n_bits, int layout);

/* As mickey_generate into a HOST buffer (pinned memory gives full copy
 * speed).  Generation runs in chunks on the device and each chunk is copied
 * back while the next one is generated.  Returns after the data is in
 * `host_out`.  Extra errors: MICKEY_E_OOM for the staging buffers. */
MICKEY_API int mickey_generate_host(mickey_streams *s, uint64_t n_bits, void *host_out,
                         int layout);

/* Wait for the handle's stream; report a device-side error if one was
 * raised (MICKEY_E_IVLEN, MICKEY_E_TIMEOUT) or a CUDA error. */
MICKEY_API int mickey_sync(mickey_streams *s);

MICKEY_API size_t mickey_num_streams(const mickey_streams *s);
/* Keystream bits generated so far by instance i (UINT64_MAX if i >= n). */
MICKEY_API uint64_t mickey_position(const mickey_streams *s, size_t i);

/* --------------------------------------------------------------------------
 * Checkpoint / resume.  A stream's state is 26 bytes: r0..r99 in bytes
 * 0..12 then s0..s99 in bytes 13..25, bit i of a register at bit (7 - i%8)
 * of byte i/8 of its half; unused low bits of bytes 12 and 25 are zero.
 * ------------------------------------------------------------------------ */

/* Copy every stream's state (n x 26 bytes) and position (n x uint64) to
 * host buffers; synchronises the handle's stream.  positions may be NULL. */
MICKEY_API int mickey_export_state(mickey_streams *s, uint8_t *states,
                        uint64_t *positions);

/* New handle from host states/positions written by mickey_export_state;
 * positions may be NULL (all 0).  Errors as mickey_init_streams_ex. */
MICKEY_API mickey_streams *mickey_import_state(const uint8_t *states,
                                    const uint64_t *positions, size_t n,
                                    void *cuda_stream);

/* --------------------------------------------------------------------------
 * Launch configuration and autotuning of the keystream kernel (per layout).
 *   mode    MICKEY_MODE_GRID: one thread per 32-lane group, clocking and
 *           emitting, 4 warps per block;
 *           MICKEY_MODE_PERSISTENT: per SM sub-partition a clock warp paired
 *           with an emission warp that transposes and stores its tiles; with
 *           at least as many 1024-instance warp-groups as clock warps the
 *           groups x tiles work line is cut into equal segments (one block
 *           per SM, cooperative), else each pair takes one whole warp-group;
 *           MICKEY_MODE_PERSISTENT2: two warps per SM sub-partition, each
 *           clocking and emitting (two blocks per SM, rows staged four
 *           tiles deep; with too few warp-groups it runs as PERSISTENT);
 *           MICKEY_MODE_AUTO: as PERSISTENT.
 *   unroll  clocks per inner step, 2 or 4.
 *   stage   the output tile of the row layouts: 0 writes each 32-clock tile's
 *           4 bytes per row directly; otherwise each row's words of several
 *           tiles are staged in shared memory and written as one chunk of
 *           4 x depth bytes -- 1: the mode's default depth (8 tiles for
 *           PERSISTENT, 4 for GRID and PERSISTENT2); 2, 4, 8: that depth
 *           (PERSISTENT: 2, 4 or 8; GRID: 2 or 4; PERSISTENT2: 4).  Used when
 *           n_bits is a multiple of 32 x depth and the output 16-byte
 *           aligned, else the row stores are direct.
 * Environment, read when a handle is created: MICKEY_MODE (grid,
 * persistent, persistent2), MICKEY_UNROLL (2, 4), MICKEY_STAGE (0, 1) and
 * MICKEY_PERSIST_BLOCKS (fewer persistent blocks than SMs) set the defaults
 * (MICKEY_STAGE takes 0, 1, 2, 4 or 8 as above);
 * MICKEY_SPIN_LIMIT bounds a persistent tail piece's wait for its head
 * (polls of about 256 ns, default 2^24), after which mickey_sync reports
 * MICKEY_E_TIMEOUT and that call's output and state are undefined;
 * MICKEY_TEST_UNPUBLISHED=1 is a test hook that makes every such wait run
 * out (tails wait for a value no head writes), to exercise that path
 * without a fault.
 * ------------------------------------------------------------------------ */
#define MICKEY_MODE_AUTO 0
#define MICKEY_MODE_GRID 1
#define MICKEY_MODE_PERSISTENT 2
#define MICKEY_MODE_PERSISTENT2 3

typedef struct {
  int mode, unroll, stage; /* stage: 0 direct, else the staging depth in tiles */
  float ms;                /* best of two timed launches */
} mickey_tune_result;

MICKEY_API int mickey_set_config(mickey_streams *s, int layout, int mode, int unroll,
                                 int stage);
MICKEY_API int mickey_get_config(const mickey_streams *s, int layout, int *mode,
                                 int *unroll, int *stage);

/* Time every configuration (mode x unroll x output tile: up to 20
 * candidates) on this handle's own streams for one call of
 * n_bits in `layout` (the state is saved and restored: positions do not
 * move), keep the fastest for that layout (among candidates within 1 % of
 * it, the one with the deepest row staging, which moves the fewest DRAM
 * bytes), and report each candidate in
 * results[0 .. min(max_results, *n_results)).  Synchronous; allocates a
 * temporary output buffer and a state copy.  results/n_results may be NULL. */
MICKEY_API int mickey_tune(mickey_streams *s, uint64_t n_bits, int layout,
                           mickey_tune_result *results, int max_results, int *n_results);

/* --------------------------------------------------------------------------
 * Batched generation: n streams, each with its own keystream length and IV
 * length, generated in one persistent launch (loading, preclocks and
 * keystream captured once as a CUDA graph, replayed by every run).  Streams
 * are packed into 32-lane groups longest first; warps take 32 groups at a
 * time from an atomic work queue in that order (longest processing time
 * first).  Output: stream i's keystream as row-major bytes (layout 1) of
 * ceil(n_bits[i] / 8) bytes at byte offset offsets[i] of `out`, offsets in
 * the caller's order, each 16-byte aligned; bytes between rows are not
 * written.
 * ------------------------------------------------------------------------ */
typedef struct mickey_batch mickey_batch;

/* Plan a batch for host arrays iv_lens (NULL = 80 each) and n_bits
 * (0 .. 2^40 each); allocates the device buffers and captures the graph on
 * the stream's device.  NULL on error (mickey_last_error: MICKEY_E_ARG,
 * MICKEY_E_IVLEN, MICKEY_E_LIMIT, MICKEY_E_OOM, MICKEY_E_CUDA). */
MICKEY_API mickey_batch *mickey_batch_create(const uint32_t *iv_lens, const uint64_t *n_bits,
                                             size_t n, void *cuda_stream);
/* Total bytes the output buffer must hold. */
MICKEY_API size_t mickey_batch_output_bytes(const mickey_batch *b);
/* Byte offset of each stream's keystream in the output (n values). */
MICKEY_API int mickey_batch_offsets(const mickey_batch *b, uint64_t *offsets);
/* Clocks of the longest group (a lower bound on the run's critical path)
 * and the sum over groups (the work); either pointer may be NULL. */
MICKEY_API int mickey_batch_clocks(const mickey_batch *b, uint64_t *max_clocks,
                                   uint64_t *total_clocks);
/* Generate every stream of the batch: keys and ivs (n x 10 bytes each, in
 * `mem`: MICKEY_MEM_HOST or MICKEY_MEM_DEVICE) are copied in, then the graph
 * is launched on the batch's stream; `out` is a device buffer of
 * mickey_batch_output_bytes bytes.  Asynchronous. */
MICKEY_API int mickey_batch_run(mickey_batch *b, const void *keys, const void *ivs, void *out,
                                int mem);
/* Launch configuration of the batch's keystream kernel: clocks per inner
 * step (2 or 4), resident blocks of 4 warps per SM (1 or 2), and
 * split_clocks: groups needing more clocks than this are each run by a whole
 * warp (lane j clocks register bits 4j..4j+3, about ten times less time per
 * clock, for long streams whose sequential clocks bound the run); 0 disables
 * the split path.  Re-captures the graph. */
MICKEY_API int mickey_batch_set_config(mickey_batch *b, int unroll, int blocks_per_sm,
                                       uint64_t split_clocks);
/* Where the split groups run (re-captures the graph):
 *   MICKEY_BATCH_SPLIT_SHARED (default): in the persistent kernel's warps,
 *     before its thread items; a long split warp keeps its SM sub-partition
 *     to itself (the shortest critical path for one batch);
 *   MICKEY_BATCH_SPLIT_OWN: in a kernel of one-warp blocks beside the thread
 *     kernel (parallel graph branches), so blocks of short thread items
 *     retire and free their registers while the split warps run on (batches
 *     back to back on several CUDA streams).
 * mickey_batch_get_split_mode returns the mode (or MICKEY_E_ARG). */
#define MICKEY_BATCH_SPLIT_SHARED 0
#define MICKEY_BATCH_SPLIT_OWN 1
MICKEY_API int mickey_batch_set_split_mode(mickey_batch *b, int mode);
MICKEY_API int mickey_batch_get_split_mode(const mickey_batch *b);
/* split_clocks / split_groups may be NULL. */
MICKEY_API int mickey_batch_get_config(const mickey_batch *b, int *unroll, int *blocks_per_sm,
                                       uint64_t *split_clocks, uint32_t *split_groups);
/* Wait for the batch's stream; MICKEY_E_IVLEN if the device saw a bad IV
 * length. */
MICKEY_API int mickey_batch_sync(mickey_batch *b);
MICKEY_API void mickey_batch_free(mickey_batch *b);

/* --------------------------------------------------------------------------
 * Serving: continuous batching over resident streams.  The server keeps one
 * 200-bit state row per stream id in device memory, so a follow-up request
 * of a stream continues its keystream without reloading the key and IV.  A
 * host scheduler (paper_1909_04750_gb300/serve.py) admits requests, packs
 * the active ones into 32-lane groups and issues steps; each step is one
 * launch that gathers the groups' states from the table, clocks them and
 * writes each request's bytes to its own buffer, then scatters the states
 * back.  Row format: words 0..3 hold R, words 4..7 hold S, register bit i at
 * bit (31 - i % 32) of word i / 32 of its half.
 * ------------------------------------------------------------------------ */
typedef struct mickey_server mickey_server;

/* Table of max_streams rows; up to max_groups groups per step.  NULL on
 * error (mickey_last_error). */
MICKEY_API mickey_server *mickey_server_create(size_t max_streams, uint32_t max_groups,
                                               void *cuda_stream);
/* Key/IV loading and preclocks of n new streams (host keys, ivs: n x 10
 * bytes; iv_lens: n values or NULL = 80); their states go to table rows
 * stream_ids[i].  Asynchronous, ordered before the next step. */
MICKEY_API int mickey_server_init_streams(mickey_server *s, const uint32_t *stream_ids,
                                          const uint8_t *keys, const uint8_t *ivs,
                                          const uint32_t *iv_lens, size_t n);
/* One step over G groups (host arrays, copied): slot_stream[32G] stream id of
 * each lane (0xffffffff: unused), slot_out[32G] device byte address where the
 * lane's bits of this step go (0: unused), group_clocks[G] bits every lane of
 * group g produces (a multiple of 8).  Groups 0..n_split-1 are each clocked
 * by a whole warp (lower time per clock, for the longest requests).
 * Asynchronous; returns after the arrays are staged. */
MICKEY_API int mickey_server_step(mickey_server *s, uint32_t G, uint32_t n_split,
                                  const uint32_t *slot_stream, const uint64_t *slot_out,
                                  const uint32_t *group_clocks);
/* Current states of the given streams in the 26-byte format of
 * mickey_export_state (synchronises). */
MICKEY_API int mickey_server_read_states(mickey_server *s, const uint32_t *stream_ids, size_t n,
                                         uint8_t *states);
/* Step kernel: clocks per inner step (2 or 4), blocks of 4 warps per SM (1 or 2). */
MICKEY_API int mickey_server_set_config(mickey_server *s, int unroll, int blocks_per_sm);
MICKEY_API int mickey_server_sync(mickey_server *s);
MICKEY_API void mickey_server_free(mickey_server *s);

/* --------------------------------------------------------------------------
 * Allocation-free key/IV loading.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory -- code
 * running inside an application whose own allocator owns the GPU's memory,
 * or a latency-bound loop that must not pay for a new allocation or for the
 * device synchronisation cudaFree implies.  It runs the same loading and
 * preclocking as mickey_init_streams, but its temporary memory is a fixed
 * array inside the library (about 3.6 MB, held on every GPU that loads the
 * library until the process exits), so it calls no allocator.
 *
 *  keys, ivs   host memory, n x 10 bytes; iv_lens host memory, n values
 *              (NULL = 80 bits each); all copied into the fixed array.
 *  n           1 .. MICKEY_NOALLOC_MAX_STREAMS.
 *  state       caller-owned DEVICE buffer of 200 * P words with
 *              P = 32 * ceil(ceil(n / 32) / 32): word w of group g at
 *              state[w * P + g] (w = 0..99: r0..r99, 100..199: s0..s99),
 *              bit l = instance 32g + l.
 *  cuda_stream the work is enqueued there; the call returns at once.
 *  Returns MICKEY_OK, MICKEY_E_ARG (NULL pointer, n == 0, n above the
 *  maximum), MICKEY_E_IVLEN, MICKEY_E_CUDA, and sets mickey_last_error()
 *  like the other calls.
 *  The first call on a device looks up the array's device address
 *  (cudaGetSymbolAddress), so make that call before any stream capture.
 *  After cudaDeviceReset the device has a new context and the array may
 *  have moved: the next call notices the new context and looks the address
 *  up again, so it too must come before any stream capture.
 *  Every call uses the same array and leaves its contents behind: calls
 *  whose work overlaps on the GPU race and must be serialised.
 * ------------------------------------------------------------------------ */
#define MICKEY_NOALLOC_MAX_STREAMS 65536
MICKEY_API int mickey_init_state_noalloc(const uint8_t *keys, const uint8_t *ivs,
                                         const uint32_t *iv_lens, size_t n, uint32_t *state,
                                         void *cuda_stream);

/* Synchronise, release all device memory of the handle.  NULL is a no-op. */
MICKEY_API void mickey_free(mickey_streams *s);

/* --------------------------------------------------------------------------
 * Errors and introspection
 * ------------------------------------------------------------------------ */
MICKEY_API int mickey_last_error(void);
MICKEY_API const char *mickey_last_error_message(void);
MICKEY_API const char *mickey_error_string(int code);

/* The five constant tables compiled into the kernels, as 100-bit masks
 * (bit i of table at word i/32, bit i%32): rows RTAPS, COMP0, COMP1, FB0,
 * FB1.  Host-only, needs no GPU. */
MICKEY_API void mickey_tables(uint32_t masks[5][4]);

/* Algorithmic 32-bit logic operations of one bitsliced CLOCK_KG of one
 * 32-lane group after constant folding into 3-input LOP3 (mixing = 0: a
 * keystream clock including z = r0 ^ s0; mixing = 1: an init clock).
 * Host-only. */
MICKEY_API int mickey_ops_per_clock(int mixing);

/* Measurement helper for the roofline: runs independent 3-input LOP3
 * chains (blocks_per_sm * SM-count blocks of `threads` threads, `iters`
 * x 128 LOP3 per thread) on the current device, synchronously.  Outputs
 * (each may be NULL): LOP3 results per SM per SM-cycle, the SM clock seen
 * (MHz), and the whole-GPU rate in 10^12 ops/s. */
MICKEY_API int mickey_probe_lop3(int blocks_per_sm, int threads, int iters,
                                 double *ops_per_sm_clk, double *sm_mhz, double *tops);

/* Measurement helper: the bare bitsliced keystream clock (z = r0 ^ s0 and
 * one CLOCK_KG, no output) of blocks_per_sm (1 or 2) * SM-count blocks of
 * 128 threads, one 32-lane group per thread, on a state of arbitrary words,
 * `clocks` clocks per group (a multiple of 4, >= 4), synchronously on the
 * current device.  Outputs (each may be NULL): algorithmic logic ops
 * (mickey_ops_per_clock(0) per group-clock) per SM per SM-cycle, and the
 * SM clock seen (MHz).  The ceiling the keystream kernel's clock can reach
 * with one (or two) warps per SM sub-partition. */
MICKEY_API int mickey_probe_clock(int blocks_per_sm, int clocks, double *ops_per_sm_clk,
                                  double *sm_mhz);

/* Library version string. */
MICKEY_API const char *mickey_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MICKEY_H */
