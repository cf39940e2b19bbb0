/*
 * bsgpu -- GB300 (sm_103a) implementation of the compression scheme of
 * Masui et al., "A compression scheme for radio data in high performance
 * computing" (arXiv:1503.00638): noise-relative precision reduction
 * (Sec. 3), Bitshuffle (Sec. 4.2) and per-block LZ4 (Sec. 4.1, 4.2.1), and
 * the inverse path.
 *
 * Conventions for every entry point below:
 *  - Pointers named d_* / in / out / ws are DEVICE pointers owned by the
 *    caller.  The library never allocates device or host memory: scratch
 *    space ("workspace") is sized by bsgpu_workspace_size() and passed in.
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*,
 *    NULL = the legacy default stream).  Argument errors are detected on the
 *    host and returned before anything is enqueued.
 *  - Errors found on the device (a corrupt stream, a bounded wait that ran
 *    out) are written to a status word at the start of the workspace; read it
 *    with bsgpu_status() once the stream has reached that point.
 *  - Input and output buffers must not overlap, and must start on a 16-byte
 *    boundary (device allocations from cudaMalloc or PyTorch always do).
 *  - No global mutable state: calls on different streams with different
 *    workspaces may run concurrently (Sec. 2.2 asks for a thread-safe
 *    library); two in-flight calls must not share one workspace.
 */
#ifndef BSGPU_H
#define BSGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (host return values and the device status word). */
#define BSGPU_OK 0
#define BSGPU_ERR_ARG (-1)      /* bad size, element size, block size or null pointer   */
#define BSGPU_ERR_SPACE (-2)    /* output capacity or workspace too small               */
#define BSGPU_ERR_CORRUPT (-3)  /* compressed stream fails validation                   */
#define BSGPU_ERR_CUDA (-4)     /* a CUDA runtime call failed                           */
#define BSGPU_ERR_TIMEOUT (-5)  /* a bounded device-side wait gave up                   */
#define BSGPU_ERR_ALIGN (-6)    /* a buffer does not start on a 16-byte boundary        */

/* Operations for bsgpu_workspace_size(). */
#define BSGPU_OP_COMPRESS 1
#define BSGPU_OP_DECOMPRESS 2
#define BSGPU_OP_COMPRESS_VIS 3
#define BSGPU_OP_REDUCE_PRECISION 4

/* Data types of a visibility cube (the _ex entry points). */
#define BSGPU_VIS_F32 0  /* interleaved float32 (re, im): complex64            */
#define BSGPU_VIS_I32 1  /* interleaved int32 (re, im), as correlators emit   */

/* Flags of the _ex entry points. */
#define BSGPU_VIS_COMPENSATE 1    /* Sec. 3.2: per-sample compensated f, see below   */
#define BSGPU_VIS_TIME_SLOWEST 2  /* input in the instrument's order, see below     */
#define BSGPU_VIS_FULL_COV 4      /* Sec. 3.1 full covariance (small arrays), below */

/* Library version string. */
const char *bsgpu_version(void);

/* Worst-case size in bytes of the framed stream that bsgpu_compress()
 * produces for n_elem elements of elem_size bytes in blocks of block_elems
 * elements (0 = the paper's default block of 4096 bytes, Sec. 4.2.1).
 * Framing (a reading of the paper, which fixes none): 8-byte big-endian
 * uncompressed byte count, 4-byte big-endian block size in bytes, then per
 * block a 4-byte big-endian compressed length and the LZ4 block, then the
 * (n_elem mod 8) trailing elements verbatim.  Returns 0 for bad arguments. */
size_t bsgpu_compress_bound(size_t n_elem, size_t elem_size, size_t block_elems);

/* Number of blocks the stream holds: full blocks of block_elems elements plus
 * one shortened block of the remaining elements rounded down to a multiple
 * of 8 (when that is not zero).  Size of the optional block-offset index. */
size_t bsgpu_num_blocks(size_t n_elem, size_t elem_size, size_t block_elems);

/* Device workspace bytes needed by bsgpu_compress (op = BSGPU_OP_COMPRESS)
 * or bsgpu_decompress (BSGPU_OP_DECOMPRESS) for these arguments; 0 for bad
 * arguments.  The workspace starts with the device status word. */
size_t bsgpu_workspace_size(int op, size_t n_elem, size_t elem_size, size_t block_elems);

/* Device workspace bytes needed by bsgpu_compress_vis (BSGPU_OP_COMPRESS_VIS)
 * or bsgpu_reduce_precision_c64 (BSGPU_OP_REDUCE_PRECISION) for a cube of
 * n_freq x n_inputs (n_inputs + 1) / 2 x n_time complex64 samples; it holds
 * the table of autocorrelations and of product indices.  block_elems as for
 * bsgpu_compress (ignored by BSGPU_OP_REDUCE_PRECISION).  0 for bad arguments. */
size_t bsgpu_vis_workspace_size(int op, int64_t n_freq, int64_t n_inputs, int64_t n_time,
                                size_t block_elems);

/* As bsgpu_vis_workspace_size, for bsgpu_compress_vis_ex (elem_size 4 or 8)
 * and bsgpu_reduce_precision_ex (elem_size ignored) with these flags (the
 * compensated f needs one more float per (freq, time) sample).  The data type
 * does not change the size.  0 for bad arguments. */
size_t bsgpu_vis_workspace_size_ex(int op, int64_t n_freq, int64_t n_inputs, int64_t n_time,
                                   size_t elem_size, size_t block_elems, int flags);

/* Read the device status word of a workspace: waits for `stream`, then
 * copies the word to *status (BSGPU_OK or a negative BSGPU_ERR_*).  Returns
 * BSGPU_OK, or BSGPU_ERR_CUDA if the copy itself failed. */
int bsgpu_status(const void *ws, void *stream, int *status);

/* Sec. 3 (Eq. rad_simple, Eq. noise, Eq. trunc_error) and Sec. 6 steps 1-3:
 * noise-relative precision reduction of a visibility cube.
 *   in, out : [n_freq][n_prod][n_time] complex64 (interleaved float32 re, im),
 *             time fastest; n_prod = n_inputs (n_inputs + 1) / 2 products in
 *             upper-triangle row-major order (0,0),(0,1)..(0,n-1),(1,1),...
 *   N       : samples per integration (Eq. rad_simple), > 0
 *   f       : maximum fractional increase of the noise variance, >= 0
 *             (f = 0 leaves the data unchanged)
 * Each real and imaginary part x of V_ij is rounded to the nearest multiple
 * of g = 2^k, ties to even, where g is the largest power of two with
 * g^2 < q = 12 f s^2; s^2 = V_ii V_jj / (2N) for i != j and V_ii^2 / N for
 * the real part of an autocorrelation, whose imaginary part is left alone.
 * q is evaluated in float32 as (fl(6f/N) * A_i) * A_j (autos:
 * (2 fl(6f/N) * A_i) * A_i) from the UNROUNDED autos A_i = Re V_ii; no
 * rounding where q is not a positive normal float.  Out of place only.
 * ws: bsgpu_vis_workspace_size(BSGPU_OP_REDUCE_PRECISION, ...) bytes. */
int bsgpu_reduce_precision_c64(const void *in, void *out, int64_t n_freq, int64_t n_inputs,
                               int64_t n_time, double N, double f, void *ws, size_t ws_bytes,
                               void *stream);

/* bsgpu_reduce_precision_c64 generalised (Sec. 3.2):
 *   dtype : BSGPU_VIS_F32, or BSGPU_VIS_I32 for a cube of int32 (re, im)
 *           pairs (same layout).  An int32 component is rounded to the
 *           nearest multiple of g = 2^k, ties to the even multiple; k <= 0
 *           (a granularity of one or less) leaves it alone, and a multiple
 *           beyond INT32_MAX is replaced by the one below it.  q is formed
 *           from the autos converted to float32 (round to nearest).
 *   flags : 0, or BSGPU_VIS_COMPENSATE: the rounding noise adds to the
 *           correlated noise of two inputs, which raises the noise of
 *           products built from them; Sec. 3.2 bounds that increase by
 *           using f m instead of f at each (freq, time) sample, where
 *           m = min over cross products i != j of 1 - |V_ij|^2 / (V_ii V_jj)
 *           (one minus the squared correlation coefficient), evaluated in
 *           float32 with each operation rounded (|V_ij|^2 as re*re + im*im),
 *           a negative or undefined value counting as 0, and m = 1 with one
 *           input.  c is then fl32(6 (f m) / N) with f m, 6 (f m) and the
 *           quotient in fp64.
 *           BSGPU_VIS_TIME_SLOWEST: `in` holds the cube in the order an
 *           instrument writes it, [n_time][n_freq][n_prod] samples (time
 *           slowest); the output is time-fastest as always.  Sec. 2 argues
 *           for a post-acquisition reorder to time-fastest (the order of
 *           reading, and the order in which neighbouring values correlate);
 *           this flag fuses that reorder into the rounding (and, in
 *           bsgpu_compress_vis_ex, into the compression).
 *           BSGPU_VIS_FULL_COV (n_inputs <= 16; not with COMPENSATE): the
 *           noise of Eq. noise from the full covariance of Eq.
 *           rad_full1-3 instead of Eq. rad_simple: for every (freq, time)
 *           sample the n^2 components left after the redundancy removal of
 *           Sec. 3.1 (Re of every product, Im of every cross product) get
 *           s^2 = 1 / (C^-1)_kk in fp64, where C^-1 is the Fisher
 *           information N tr(E_a W E_b W) of the components (W = V^-1):
 *           (C^-1)_kk = N W_ii^2 for Re V_ii and 2 N (W_ii W_jj +- Re(W_ij^2))
 *           for Re / Im V_ij, from an n x n complex Cholesky factorisation
 *           per sample; q = fl32(12 f s^2).  A sample whose C is not
 *           positive definite (V neither positive nor negative definite) is
 *           left unrounded.  Sec. 3.1 keeps this to arrays of a few dozen
 *           inputs at most; the workspace holds one float per component.
 * ws: bsgpu_vis_workspace_size_ex(BSGPU_OP_REDUCE_PRECISION, ..., flags). */
int bsgpu_reduce_precision_ex(const void *in, void *out, int dtype, int64_t n_freq,
                              int64_t n_inputs, int64_t n_time, double N, double f, int flags,
                              void *ws, size_t ws_bytes, void *stream);

/* Eq. noise with the full covariance of Eq. rad_full1-3 (Sec. 3.1), on its
 * own: d_s2 receives [n_freq][n_time][n_inputs^2] fp64 unmarginalized
 * variances s^2 = 1/(C^-1)_kk in the component order of BSGPU_VIS_FULL_COV
 * (0 for a sample whose C is not positive definite).  flags: 0 or
 * BSGPU_VIS_TIME_SLOWEST.  n_inputs <= 16.  ws:
 * bsgpu_vis_workspace_size_ex(BSGPU_OP_REDUCE_PRECISION, ..., flags |
 * BSGPU_VIS_FULL_COV). */
int bsgpu_full_noise_var(const void *vis, int dtype, int64_t n_freq, int64_t n_inputs,
                         int64_t n_time, double N, int flags, double *d_s2, void *ws,
                         size_t ws_bytes, void *stream);

/* Sec. 2: the post-acquisition reorder on its own.  in holds n_time rows of
 * n_series elements of elem_size (1, 2, 4 or 8) bytes (time slowest); out
 * receives n_series rows of n_time elements (time fastest): out[s][t] =
 * in[t][s].  A complex64 visibility cube is n_series = n_freq n_prod
 * elements of 8 bytes.  Buffers aligned to elem_size, not overlapping. */
int bsgpu_reorder_time(const void *in, void *out, uint64_t n_time, uint64_t n_series,
                       size_t elem_size, void *stream);

/* Sec. 4.2 and Sec. 6 step 4: Bitshuffle.  Within each block of block_elems
 * elements (a multiple of 8; 0 = 4096 bytes), bit r of element e (r = 8 *
 * byte + bit of the little-endian element, bit 0 = least significant) moves
 * to byte r * (block_elems / 8) + e / 8, bit e % 8.  A trailing partial block
 * is shortened to a multiple of 8 elements and transposed the same way; the
 * last (n_elem mod 8) elements are copied unchanged.  elem_size is 1, 2, 4
 * or 8.  in and out hold n_elem * elem_size bytes. */
int bsgpu_bitshuffle(const void *in, void *out, size_t n_elem, size_t elem_size,
                     size_t block_elems, void *stream);

/* Inverse of bsgpu_bitshuffle with the same arguments. */
int bsgpu_bitunshuffle(const void *in, void *out, size_t n_elem, size_t elem_size,
                       size_t block_elems, void *stream);

/* Sec. 4.2.1 and Sec. 6 steps 4-5: Bitshuffle each block and compress it
 * with LZ4 while it is on chip, writing the framed stream described at
 * bsgpu_compress_bound().
 *   in              : n_elem * elem_size bytes
 *   level           : LZ4 match search.  0: matches of 8 or more bytes
 *                     against the same column of the previous bit-row and
 *                     runs (fastest to encode and to decode); 1: also a hash
 *                     table of earlier positions (better ratio on data with
 *                     other repeats, slower).
 *   out, out_cap    : at least bsgpu_compress_bound() bytes
 *   d_out_bytes     : device uint64, receives the stream length
 *   d_block_offsets : NULL, or bsgpu_num_blocks() device uint64s that
 *                     receive the byte offset of each block's length field
 *                     (lets bsgpu_decompress() start every block at once)
 * Block sizes up to 65536 bytes (LZ4 offsets are 16-bit).  The LZ4 encoding
 * is deterministic but is not byte-identical to other encoders' (LZ4 output
 * is not unique); any conforming LZ4 block decoder reads it. */
int bsgpu_compress(const void *in, size_t n_elem, size_t elem_size, size_t block_elems, int level,
                   void *out, size_t out_cap, uint64_t *d_out_bytes, uint64_t *d_block_offsets,
                   void *ws, size_t ws_bytes, void *stream);

/* Inverse of bsgpu_compress: decode in_bytes of framed stream into n_elem
 * elements.  d_block_offsets is the index written by bsgpu_compress (or
 * NULL: the block chain is then walked on the device by one thread first,
 * which is slow for large streams).  A stream whose header does not match
 * (n_elem, elem_size, block_elems), or that fails LZ4 validation (offset 0
 * or before the block start, a length running past either buffer, a block
 * that does not decode to exactly its size), sets BSGPU_ERR_CORRUPT in the
 * status word; the output is then unspecified but nothing outside the given
 * buffers is touched. */
int bsgpu_decompress(const void *in, size_t in_bytes, void *out, size_t n_elem, size_t elem_size,
                     size_t block_elems, const uint64_t *d_block_offsets, void *ws,
                     size_t ws_bytes, void *stream);

/* Sec. 6 steps 1-5 fused: precision reduction of a visibility cube (as in
 * bsgpu_reduce_precision_c64) followed by Bitshuffle + LZ4 of the rounded
 * float32 values (elem_size 4), in one pass over the input.  The stream is
 * the one bsgpu_compress() would write for the rounded cube viewed as
 * 2 * n_freq * n_prod * n_time float32 elements; decode it with
 * bsgpu_decompress(elem_size = 4).  level as for bsgpu_compress.
 * ws: bsgpu_vis_workspace_size(BSGPU_OP_COMPRESS_VIS, ...) bytes. */
int bsgpu_compress_vis(const void *vis, int64_t n_freq, int64_t n_inputs, int64_t n_time,
                       double N, double f, size_t block_elems, int level, void *out,
                       size_t out_cap,
                       uint64_t *d_out_bytes, uint64_t *d_block_offsets, void *ws,
                       size_t ws_bytes, void *stream);

/* bsgpu_compress_vis generalised: dtype and flags as for
 * bsgpu_reduce_precision_ex; elem_size 4 compresses the rounded cube as
 * 2 n_freq n_prod n_time 4-byte components, elem_size 8 as n_freq n_prod
 * n_time 8-byte (re, im) samples (the bit-rows then interleave the two
 * components' bits, Sec. 4.2).  Decode with bsgpu_decompress(elem_size).
 * ws: bsgpu_vis_workspace_size_ex(BSGPU_OP_COMPRESS_VIS, ..., elem_size,
 * block_elems, flags) bytes. */
int bsgpu_compress_vis_ex(const void *vis, int dtype, int64_t n_freq, int64_t n_inputs,
                          int64_t n_time, double N, double f, int flags, size_t elem_size,
                          size_t block_elems, int level, void *out, size_t out_cap,
                          uint64_t *d_out_bytes, uint64_t *d_block_offsets, void *ws,
                          size_t ws_bytes, void *stream);

/* bsgpu_compress for callers that cannot allocate device memory (the paper
 * has no counterpart: this is a deployment variant).  Such callers are handed
 * buffers but may not allocate: a filter callback of an I/O library receives
 * only the chunk's input and output buffers; a real-time acquisition loop
 * allocates everything at start-up and must not call cudaMalloc afterwards,
 * since it synchronizes the device; a process whose device memory is wholly
 * owned by a pool.
 *   Arguments and output as for bsgpu_compress, without the workspace.  The
 *   scratch (status word, tile counter, 8 bytes of look-back state per block)
 *   lives in a fixed array inside the library of 256 + 8 * 131072 bytes
 *   (about 1 MiB), held in every context the library's module is loaded
 *   into (each device the process uses it on) until the process exits; inputs of more than 131072 blocks (1 GiB at 8 KiB blocks)
 *   are rejected with BSGPU_ERR_SPACE before anything is enqueued.
 *   The first call in each context (the device's primary context, or any
 *   other context the caller makes current) looks up the array's device
 *   address with that context current and caches it for that context.  With
 *   lazy module loading (the CUDA default) that first call also loads the
 *   library's module into the context, which places the array and may
 *   synchronize the device: make it at start-up, as a warm-up, before any
 *   stream capture (or set CUDA_MODULE_LOADING=EAGER to do it when the
 *   library is loaded).  Later calls allocate and free nothing and call no
 *   allocating routine.
 *   Every call shares the one array: calls that overlap on the GPU (on
 *   different streams, or from different threads) race and corrupt each
 *   other's output; serialize them.
 *   Any device-side failure (a bounded wait that ran out, or any other
 *   error the kernels record) is reported by writing 0 to *d_out_bytes (a
 *   valid stream is at least 12 bytes long); the call's own return value
 *   covers argument and launch errors only. */
int bsgpu_compress_noalloc(const void *in, size_t n_elem, size_t elem_size, size_t block_elems,
                           int level, void *out, size_t out_cap, uint64_t *d_out_bytes,
                           uint64_t *d_block_offsets, void *stream);

/* ------------------------------------------------------------------------
 * Batched codec (Sec. 4.2.1: blocks are independent units of work).  Many
 * independent chunks -- each its own framed stream, with its own element
 * size (1, 2, 4 or 8) and block size (at most 8192 bytes) -- compressed or
 * decompressed by ONE persistent launch whose work queue runs over every
 * (chunk, block) item, so uneven chunk sizes do not leave SMs idle.  Each
 * chunk's stream is byte-identical to what bsgpu_compress() writes for that
 * chunk alone with the same level.
 * ------------------------------------------------------------------------ */

/* One chunk of a batch (host memory; pointers are device pointers, 16-byte
 * aligned).
 *   compress  : in = n_elem * elem_size bytes; out = stream buffer of
 *               out_cap >= bsgpu_compress_bound() bytes; in_bytes ignored.
 *   decompress: in = the chunk's stream of in_bytes bytes (or see
 *               d_in_bytes); out = n_elem * elem_size bytes; out_cap ignored.
 *   block_elems: a multiple of 8 with block_elems * elem_size <= 8192, or 0
 *               for the 4096-byte default.
 *   block_offsets: NULL, or the chunk's own block index (bsgpu_num_blocks()
 *               device uint64s, 8-byte aligned): written by a compress batch,
 *               read by a decompress batch, in place of the batch-wide index
 *               argument (a stream kept with its index needs no chain walk). */
typedef struct bsgpu_chunk {
    const void *in;
    void *out;
    uint64_t n_elem;
    uint64_t in_bytes;
    uint64_t out_cap;
    uint32_t elem_size;
    uint32_t block_elems;
    uint64_t *block_offsets;
} bsgpu_chunk;

/* Bytes of the table image for n_chunks chunks (0 for none). */
size_t bsgpu_batch_table_bytes(uint32_t n_chunks);

/* Host-only: validate the chunks for op (BSGPU_OP_COMPRESS or
 * BSGPU_OP_DECOMPRESS) and write the table image (bsgpu_batch_table_bytes
 * bytes) to host memory `table`; the caller copies it, unchanged, to 16-byte
 * aligned device memory before the batch call (it holds the chunks' device
 * pointers, sizes and first item indices).  *n_items receives the number of
 * items: each chunk's block count, or 1 for a chunk of fewer than 8 elements.
 * *ws_bytes receives the device workspace the batch call needs.  Chunk c's
 * block index entries start at item (sum over earlier chunks of their item
 * counts).  Errors: BSGPU_ERR_ARG (element size, block size, null pointer),
 * BSGPU_ERR_ALIGN, BSGPU_ERR_SPACE (table or a chunk's out_cap too small). */
int bsgpu_batch_plan(int op, const bsgpu_chunk *chunks, uint32_t n_chunks, void *table,
                     size_t table_bytes, uint64_t *n_items, size_t *ws_bytes);

/* Compress every chunk of a planned batch.
 *   d_table         : the device copy of the table image
 *   level           : as for bsgpu_compress
 *   d_out_bytes     : n_chunks device uint64s, each chunk's stream length
 *   d_block_offsets : NULL or n_items device uint64s (per-chunk block index,
 *                     offsets relative to the chunk's stream)
 *   d_chunk_status  : n_chunks device ints, zeroed by the call, then
 *                     BSGPU_ERR_SPACE / BSGPU_ERR_TIMEOUT for a chunk that
 *                     failed on the device
 *   ctas_per_sm     : resident one-warp CTAs per SM (0 = as many as fit;
 *                     the tuning knob of the batch engine)
 * Asynchronous on `stream`; nothing allocated. */
int bsgpu_compress_batch(const void *d_table, uint32_t n_chunks, uint64_t n_items, int level,
                         uint64_t *d_out_bytes, uint64_t *d_block_offsets, int *d_chunk_status,
                         void *ws, size_t ws_bytes, uint32_t ctas_per_sm, void *stream);

/* Decompress every chunk of a planned batch (planned with
 * BSGPU_OP_DECOMPRESS).  d_in_bytes: NULL (use each chunk's in_bytes) or
 * n_chunks device uint64s of stream lengths (e.g. a compress batch's
 * d_out_bytes, so both can run back to back without the host).
 * d_block_offsets: the index from bsgpu_compress_batch, or NULL (each
 * chunk's block chain is then walked on the device by one thread per chunk
 * first: slow for long chunks).  A corrupt chunk sets BSGPU_ERR_CORRUPT in
 * its d_chunk_status entry; its output is then unspecified, the other
 * chunks are unaffected and nothing outside the given buffers is touched. */
int bsgpu_decompress_batch(const void *d_table, uint32_t n_chunks, uint64_t n_items,
                           const uint64_t *d_in_bytes, const uint64_t *d_block_offsets,
                           int *d_chunk_status, void *ws, size_t ws_bytes, uint32_t ctas_per_sm,
                           void *stream);

/* The batch calls with a second launch-shape knob (Sec. 4.2.1: blocks are
 * the independent units of work, the launch shape only decides how many
 * are in flight): warps_per_cta of 1, 2 or 4 warps per CTA, each warp an
 * independent worker with its own shared-memory slice; ctas_per_sm then
 * counts CTAs of that many warps (0 = as many as fit).  The output is the
 * same for every shape.  bsgpu_compress_batch / bsgpu_decompress_batch are
 * these with warps_per_cta = 1.  BSGPU_ERR_ARG for any other warps_per_cta;
 * otherwise as the calls above. */
int bsgpu_compress_batch_ex(const void *d_table, uint32_t n_chunks, uint64_t n_items, int level,
                            uint64_t *d_out_bytes, uint64_t *d_block_offsets, int *d_chunk_status,
                            void *ws, size_t ws_bytes, uint32_t ctas_per_sm,
                            uint32_t warps_per_cta, void *stream);
int bsgpu_decompress_batch_ex(const void *d_table, uint32_t n_chunks, uint64_t n_items,
                              const uint64_t *d_in_bytes, const uint64_t *d_block_offsets,
                              int *d_chunk_status, void *ws, size_t ws_bytes,
                              uint32_t ctas_per_sm, uint32_t warps_per_cta, void *stream);

/* ------------------------------------------------------------------------
 * Offset allocator for a fixed device arena (host only; the paper has no
 * counterpart: it serves the admission control of a server that keeps one
 * device allocation of a fixed capacity and gives byte ranges of it to the
 * requests it admits).  Best fit, neighbouring free ranges merged on free,
 * every range a multiple of `align` long and aligned to it.  Thread-safe.
 * Nothing here touches device memory.
 * ------------------------------------------------------------------------ */

/* A new arena of capacity bytes (rounded down to a multiple of align, a power
 * of two); NULL for bad arguments or no host memory. */
void *bsgpu_arena_create(uint64_t capacity, uint64_t align);
void bsgpu_arena_destroy(void *arena);

/* Reserve `bytes` (rounded up to align; 0 counts as 1): *offset receives the
 * range's start.  BSGPU_ERR_SPACE when no free range is large enough (the
 * arena is unchanged), BSGPU_ERR_ARG for a null argument. */
int bsgpu_arena_alloc(void *arena, uint64_t bytes, uint64_t *offset);

/* Release the range starting at offset; BSGPU_ERR_ARG if none starts there. */
int bsgpu_arena_free(void *arena, uint64_t offset);

/* Bytes reserved now, the largest free range, the most bytes ever reserved
 * at once, and the number of free ranges (any pointer may be NULL). */
int bsgpu_arena_stats(const void *arena, uint64_t *used_bytes, uint64_t *largest_free,
                      uint64_t *high_water, uint64_t *n_free_ranges);

#ifdef __cplusplus
}
#endif

#endif /* BSGPU_H */
