// Kernel argument blocks and launcher declarations shared by the kernel
// translation units and the C-ABI layer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace bsg {

// Visibility-cube geometry for the precision reduction (Sec. 3).
struct VisParams {
    const float *autos;     // [n_freq][n_in][n_time] unrounded Re V_ii
    const uint32_t *pairs;  // [n_prod]: i | (j << 16), upper-triangle row-major
    uint32_t n_in, T, P;    // inputs, time samples, products
    uint32_t qT, rT;        // 32 / T and 32 % T (advance of a lane by 32 samples)
    float c, c2;            // fl32(6 f / N) and 2 c
    const float *cft;       // per (freq, time) compensated c (Sec. 3.2), or null
    int is_int;             // components are int32 (else float32)
    int tslow;              // the input is time-slowest: [T][n_freq n_prod] samples
    uint32_t FP;            // n_freq n_prod (series of T samples)
    const float *qtab;      // full-covariance q per component [n_freq][M][T], or null
    uint32_t M;             // components per sample (n_in^2) when qtab is set
    FastDiv dT, dP;         // division by T and by P
    int enabled;
};

// Full-covariance q of the real (im = false) or imaginary part of product
// p = (i, j) at (f, t): components are Re of every product, then Im of every
// cross product (i + 1 autos precede (i, j) in product order).
__device__ __forceinline__ float vis_q_full(const VisParams &P, uint32_t f, uint32_t t,
                                            uint32_t p, uint32_t i, bool im)
{
    const uint32_t comp = im ? P.P + p - i - 1 : p;
    return __ldg(P.qtab + ((size_t)f * P.M + comp) * P.T + t);
}

// Input sample holding time-fastest complex index c ((f, p) series c / T,
// time c % T): the same index, or its place in a time-slowest input (the
// instrument's order before the post-acquisition reorder of Sec. 2).
__host__ __device__ __forceinline__ uint64_t vis_src(const VisParams &P, uint64_t c)
{
    return P.tslow ? (c % P.T) * P.FP + c / P.T : c;
}

// c (2c for the real part of an auto) of the sample at (f, t)
__device__ __forceinline__ float vis_c(const VisParams &P, uint32_t f, uint32_t t, bool is_auto)
{
    const float c = P.cft ? P.cft[(size_t)f * P.T + t] : P.c;
    return is_auto ? 2.0f * c : c;
}

// One framed stream (compress / decompress / bitshuffle).
struct CodecArgs {
    const uint8_t *in;
    uint8_t *out;
    uint64_t in_bytes;       // decompress: stream length
    uint64_t out_cap;        // compress: output capacity
    uint64_t *out_bytes;     // compress: stream length (device)
    uint64_t *block_offsets; // compress: written if non-null; decompress: read
    uint64_t *tile_state;    // compress: decoupled look-back state, zeroed
    uint32_t *tile_counter;  // dynamic tile counter, zeroed
    int *status;             // device status word, zeroed
    uint64_t n_elem;
    uint32_t es, B, nb, last_B, tail_elems;
    int level;               // compress: LZ4 search level (0 structural, 1 + hash)
    uint32_t tile_begin;     // compress: tiles [tile_begin, tile_end) of this launch
    uint32_t tile_end;
    uint8_t *slots;          // compress: two staging slots per warp (null: none)
    uint32_t nslot_warps;    // warps the slots cover
    VisParams vis;
};

// Shared-memory bytes per warp-CTA for each kernel family and block-size class
// (staged: the general compressor with staging slots, see launch_compress).
uint32_t compress_smem_bytes(uint32_t maxb, int level, bool staged = false);
// bytes of one staging slot of the general compressor
uint32_t compress_slot_bytes(uint32_t maxb);
uint32_t decompress_smem_bytes(uint32_t maxb);
// resident CTAs per SM of the one-buffer (in-place) decompress kernel
uint32_t decompress_inplace_blocks_per_sm(uint32_t es);
// shared memory of the in-place decompress kernel for other shapes
uint32_t decompress_inplace_any_smem_bytes(uint32_t maxb);
uint32_t shuffle_smem_bytes(uint32_t maxb);

// Launchers (return cudaGetLastError()).  `grid` warps of 32 threads.
cudaError_t launch_vis_tables(const float *vis, const VisParams &P, uint32_t n_freq,
                              cudaStream_t s);
// time-slowest [T][S] elements of es bytes -> time-fastest [S][T]
cudaError_t launch_reorder_time(const void *in, void *out, uint64_t T, uint64_t S, uint32_t es,
                                cudaStream_t s);
// full-covariance noise (Eq. rad_full1-3, Eq. noise) per (freq, time): q
// table into P.qtab and, when s2 is not null, s^2 per component [F][T][M]
// (fp64)
cudaError_t launch_full_noise(const void *vis, const VisParams &P, uint32_t n_freq, double f,
                              double N, double *s2, cudaStream_t s);
constexpr uint32_t FULL_MAX_INPUTS = 16;   // inputs of the full-covariance noise
// per (freq, time) compensated c of Sec. 3.2 into P.cft (needs the tables)
cudaError_t launch_vis_compensation(const void *vis, const VisParams &P, uint32_t n_freq,
                                    double f, double N, cudaStream_t s);
cudaError_t launch_reduce_precision(const float *in, float *out, uint64_t n_cplx,
                                    const VisParams &v, uint32_t grid, cudaStream_t s);
cudaError_t launch_shuffle(const CodecArgs &a, bool inverse, uint32_t maxb, uint32_t grid,
                           cudaStream_t s);
// General compressor, tiles [a.tile_begin, a.tile_end).  With a.slots (two
// slots of compress_slot_bytes(maxb) per CTA of the grid, grid <=
// a.nslot_warps) blocks are placed one block late from the slots; without,
// each block is placed as soon as it is encoded.
cudaError_t launch_compress(const CodecArgs &a, uint32_t maxb, uint32_t grid, cudaStream_t s);
// Fast path for full blocks that the in-place register transposes take
// (shuffle_inplace_ok; for a cube also n_time % 16 == 0): tiles
// [0, a.tile_end), placement one block late through per-warp staging slots.
cudaError_t launch_compress_fast(const CodecArgs &a, uint32_t grid, cudaStream_t s);
uint32_t compress_fast_smem_bytes(int level);
uint32_t compress_fast_blocks_per_sm(int level, uint32_t es);
// the same for a time-slowest cube (n_time % 16 == 0), in tslow.cu
cudaError_t launch_compress_fast_tslow(const CodecArgs &a, uint32_t grid, cudaStream_t s);
uint32_t compress_fast_tslow_blocks_per_sm(int level, uint32_t es);
// the same for a time-fastest cube of 4-byte components with n_time % 16 != 0
cudaError_t launch_compress_fast_ps(const CodecArgs &a, uint32_t grid, cudaStream_t s);
uint32_t compress_fast_ps_blocks_per_sm(int level);
// staging slot size of the fast path and the warp count its slots cover
constexpr uint32_t FAST_SLOT_BYTES = 8304;
constexpr uint32_t FAST_MAX_WARPS = 3072;
cudaError_t launch_compress_small(const CodecArgs &a, cudaStream_t s);
cudaError_t launch_decompress(const CodecArgs &a, uint32_t maxb, uint32_t grid, cudaStream_t s);
// In-place decoding for blocks over 8 KiB and 1-byte elements, the output
// 16-byte aligned for every block ((a.B * a.es) % 16 == 0, a.out aligned).
cudaError_t launch_decompress_inplace_any(const CodecArgs &a, uint32_t maxb, uint32_t grid,
                                          cudaStream_t s);
// Block index of a stream without one (seg_ws: SEG_WS_BYTES of workspace for
// the parallel recovery, or null for the staged serial walk alone).
constexpr size_t SEG_WS_BYTES = 256 + 160 * 2048;
cudaError_t launch_chain_walk(const CodecArgs &a, uint64_t *offsets, void *seg_ws, cudaStream_t s);

// Block-size class: the smallest supported shared-memory plan for `bytes`.
inline uint32_t maxb_class(uint32_t bytes)
{
    return bytes <= 8192 ? 8192u : (bytes <= 16384 ? 16384u : (bytes <= 32768 ? 32768u : 65536u));
}

}  // namespace bsg
