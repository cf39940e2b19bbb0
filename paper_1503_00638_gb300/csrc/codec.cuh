// Device-side building blocks shared by the codec kernels (kernels.cu) and
// the batched engine (batch.cu): shared-memory plans, bulk-copy staging and
// write-out, the precision-reduction helpers (Sec. 3.2), the decoupled
// look-back that places variable-size compressed blocks in one pass, block
// placement and encoding, and the decoder's block fetch.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.cuh"
#include "lz4_warp.cuh"
#include "shuffle.cuh"

namespace bsg {

// ---------------------------------------------------------------------------
// Shared-memory plans
// ---------------------------------------------------------------------------
__host__ __device__ constexpr uint32_t r16(uint32_t x) { return (x + 15u) & ~15u; }
__host__ __device__ constexpr uint32_t r128(uint32_t x) { return (x + 127u) & ~127u; }
__host__ __device__ constexpr uint32_t cmax(uint32_t a, uint32_t b) { return a > b ? a : b; }
__host__ __device__ constexpr uint32_t lz4b(uint32_t n) { return n + n / 255u + 16u; }

template <uint32_t MAXB, int LEVEL>
struct CompPlan {
    static constexpr uint32_t IN = r16(MAXB);          // staged block (bulk copy target)
    static constexpr uint32_t TMP = r16(MAXB + 16);    // bit-rows (LZ4 input, read 8 past)
    // LZ4 output with its 4-byte length field in front (write-out reads 16 past)
    static constexpr uint32_t OUT = r16(4 + lz4b(MAXB) + 16);
    // level 1: one 16-bit hash entry per probed word position of the largest
    // block; level 0: two word-equality bitmaps
    static constexpr int HBITS = MAXB <= 8192 ? 11 : (MAXB <= 16384 ? 12 : 13);
    static constexpr uint32_t SCR = LEVEL >= 1 ? (2u << HBITS) : 2u * 4u * (MAXB / 128u + 2u);
    static constexpr uint32_t BYTES = IN + TMP + OUT + r16(SCR) + 16;
    // staged: the LZ4 output goes to a staging slot in global memory and the
    // block is placed one block later, coming back into `tmp` and the scratch
    // after it (so no output buffer; two barriers)
    static constexpr uint32_t SLOT = r16(4 + lz4b(MAXB) + 32);
    static constexpr uint32_t BYTES_STAGED = IN + TMP + r16(SCR) + 32;
    static_assert(TMP + SCR >= r16(4 + lz4b(MAXB)), "placement buffer");
};

template <uint32_t MAXB>
struct DecPlan {
    // stream bytes of one block at their 16-byte phase, read 8 past the end
    static constexpr uint32_t COMP = r16(16 + 4 + lz4b(MAXB) + 16);
    static constexpr uint32_t DEC = r16(MAXB + 16);
    static constexpr uint32_t BYTES = COMP + DEC + 16;
};

template <uint32_t MAXB>
struct ShufPlan {
    static constexpr uint32_t BUF = r128(MAXB + 32);
    static constexpr uint32_t BYTES = 3 * BUF + 16;
};


// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
BSG_D uint32_t grab_tile(uint32_t *counter, uint32_t lane)
{
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(counter, 1u);
    return __shfl_sync(FULL, t, 0);
}

BSG_D uint32_t block_elems_of(const CodecArgs &a, uint32_t tile)
{
    return tile + 1 == a.nb ? a.last_B : a.B;
}

// Start moving `bytes` from global `src` to shared `dst`: one bulk copy when
// both ends are 16-byte aligned (returns true: wait on `bar`), otherwise a
// plain warp copy (returns false: done).
BSG_D bool load_block(uint8_t *dst, const uint8_t *src, uint32_t bytes, uint64_t *bar,
                      uint32_t lane)
{
    if ((bytes & 15u) == 0 && ((uintptr_t)src & 15u) == 0 && bytes > 0) {
        if (lane == 0) {
            mbar_arrive_expect_tx(bar, bytes);
            bulk_g2s(dst, src, bytes, bar);
        }
        return true;
    }
    for (uint32_t k = lane; k < bytes; k += 32) dst[k] = src[k];
    __syncwarp();
    return false;
}

// Block `tile` of a stream into shared `dst`: a bulk copy (returns true: wait
// on `bar`) or, for a time-slowest visibility cube, a gather of its complex
// samples into time-fastest order (8-byte loads; consecutive lanes take
// consecutive output samples, so the shared stores are conflict-free and the
// strided global reads share cache lines across a warp's successive steps).
BSG_D bool load_block_any(const CodecArgs &a, uint8_t *dst, uint32_t tile, uint64_t *bar,
                          uint32_t lane)
{
    const uint32_t bytes = block_elems_of(a, tile) * a.es;
    if (!a.vis.enabled || !a.vis.tslow)
        return load_block(dst, a.in + (uint64_t)tile * a.B * a.es, bytes, bar, lane);
    const uint64_t c0 = ((uint64_t)tile * a.B * a.es) >> 3;
    const uint2 *src = reinterpret_cast<const uint2 *>(a.in);
    uint2 *d = reinterpret_cast<uint2 *>(dst);
    for (uint32_t k = lane; k < bytes / 8; k += 32) d[k] = __ldg(src + vis_src(a.vis, c0 + k));
    __syncwarp();
    return false;
}

// Full block `tile` of a time-slowest cube ([T][F P] complex samples, T a
// multiple of 16) into shared `dst` in time-fastest order.  The block is
// groups of 16 consecutive time samples of one (freq, product) series, 128
// output bytes (eight 16-byte chunks of two samples) each; lane l takes
// groups l, l + 32, ...  Lanes run through the chunks in an order rotated by
// m = (l / 4) mod 8, so at every step the four lanes of one 32-byte sector
// of neighbouring series read the same time row (full sectors), and the
// chunks the 32 lanes store fall in eight different bank groups (no shared-
// memory conflicts).
BSG_D void gather_tslow_block(const CodecArgs &a, uint8_t *dst, uint32_t tile, uint32_t lane)
{
    const VisParams &P = a.vis;
    const uint32_t n8 = (uint32_t)(((uint64_t)a.B * a.es) >> 3);   // samples per block
    const uint32_t c0 = tile * n8;        // complex indices of a cube are below 2^32
    const uint64_t row = P.FP;            // one time step, in samples
    const uint2 *src = reinterpret_cast<const uint2 *>(a.in);
    const uint32_t m = (lane >> 2) & 7u;
    for (uint32_t q = lane; q < n8 / 16u; q += 32) {
        const uint32_t c = c0 + 16u * q, s = fastdiv(c, P.dT), t0 = c - s * P.T;
        const uint2 *p = src + (uint64_t)t0 * row + s;
        uint4 *d = reinterpret_cast<uint4 *>(dst + (size_t)128 * q);
#pragma unroll
        for (uint32_t k = 0; k < 8; k++) {
            const uint32_t x = (k + m) & 7u;   // chunk x: samples t0 + 2x, t0 + 2x + 1
            const uint2 u = __ldg(p + (uint64_t)(2 * x) * row);
            const uint2 v = __ldg(p + (uint64_t)(2 * x + 1) * row);
            d[x] = make_uint4(u.x, u.y, v.x, v.y);
        }
    }
}

// Full block `tile` of a time-slowest cube whose time axis is not a multiple
// of 16 (series of 16 samples would straddle products) into shared `dst` in
// time-fastest order, one complex sample per lane and step: output sample
// c0 + k comes from time (c0 + k) mod T of series (c0 + k) / T, the division
// through the precomputed multiply-high.
BSG_D void gather_tslow_samples(const CodecArgs &a, uint8_t *dst, uint32_t tile, uint32_t lane)
{
    const VisParams &P = a.vis;
    const uint32_t n8 = (uint32_t)(((uint64_t)a.B * a.es) >> 3);   // samples per block
    const uint32_t c0 = tile * n8;        // complex indices of a cube are below 2^32
    const uint2 *src = reinterpret_cast<const uint2 *>(a.in);
    uint2 *d = reinterpret_cast<uint2 *>(dst);
    for (uint32_t k = lane; k < n8; k += 32) {
        const uint32_t c = c0 + k, s = fastdiv(c, P.dT), t = c - s * P.T;
        d[k] = __ldg(src + (uint64_t)t * P.FP + s);
    }
}

// Copy len bytes from 16-byte aligned shared `s` to global `g` (any alignment):
// byte stores up to g's next 16-byte boundary, then 16-byte stores assembled
// from two aligned shared vectors and a funnel shift, then the ragged end.
// Reads up to 32 bytes past s + len.
BSG_D void copy_out(const uint8_t *s, uint8_t *g, uint32_t len, uint32_t lane)
{
    uint32_t head = (uint32_t)((16u - ((uintptr_t)g & 15u)) & 15u);
    if (head > len) head = len;
    if (lane < head) g[lane] = s[lane];
    const uint32_t nchunk = (len - head) / 16u;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(s);
    const uint32_t q = (head >> 2) & 3u, sh = (head & 3u) * 8u;
    for (uint32_t c = lane; c < nchunk; c += 32) {
        uint32_t so = head + 16u * c;
        uint4 A = s4[so >> 4], B = s4[(so >> 4) + 1];
        uint4 v;
        switch (q) {  // uniform across the warp
        case 0:
            v = make_uint4(funnel_r(A.x, A.y, sh), funnel_r(A.y, A.z, sh), funnel_r(A.z, A.w, sh),
                           funnel_r(A.w, B.x, sh));
            break;
        case 1:
            v = make_uint4(funnel_r(A.y, A.z, sh), funnel_r(A.z, A.w, sh), funnel_r(A.w, B.x, sh),
                           funnel_r(B.x, B.y, sh));
            break;
        case 2:
            v = make_uint4(funnel_r(A.z, A.w, sh), funnel_r(A.w, B.x, sh), funnel_r(B.x, B.y, sh),
                           funnel_r(B.y, B.z, sh));
            break;
        default:
            v = make_uint4(funnel_r(A.w, B.x, sh), funnel_r(B.x, B.y, sh), funnel_r(B.y, B.z, sh),
                           funnel_r(B.z, B.w, sh));
            break;
        }
        *reinterpret_cast<uint4 *>(g + so) = v;
    }
    for (uint32_t k = head + 16u * nchunk + lane; k < len; k += 32) g[k] = s[k];
}

BSG_D void put_be32(uint8_t *p, uint32_t v)
{
    p[0] = (uint8_t)(v >> 24);
    p[1] = (uint8_t)(v >> 16);
    p[2] = (uint8_t)(v >> 8);
    p[3] = (uint8_t)v;
}

BSG_D uint32_t get_be32(const uint8_t *p)
{
    return ((uint32_t)p[0] << 24) | ((uint32_t)p[1] << 16) | ((uint32_t)p[2] << 8) | p[3];
}

// 12-byte chunk header: big-endian total bytes, big-endian block bytes
BSG_D void write_chunk_header(uint8_t *out, uint64_t total, uint32_t block_bytes, uint32_t lane)
{
    if (lane < 8) out[lane] = (uint8_t)(total >> (8 * (7 - lane)));
    else if (lane < 12) out[lane] = (uint8_t)(block_bytes >> (8 * (11 - lane)));
}

// ---------------------------------------------------------------------------
// Precision reduction of complex samples (Sec. 3.2, Sec. 6 steps 1-3)
// ---------------------------------------------------------------------------
// Product index of (i, j), i <= j, in upper-triangle row-major order.
BSG_D uint32_t ij_prod(const VisParams &P, uint32_t i, uint32_t j)
{
    return i * P.n_in - i * (i - 1) / 2 + (j - i);
}

// Round one complex sample (re, im bits) of product p = (i, j) at (f, t).
BSG_D uint2 reduce_sample(uint2 v, uint32_t ij, uint32_t f, uint32_t t, const VisParams &P)
{
    const uint32_t i = ij & 0xffffu, j = ij >> 16;
    const bool is_auto = i == j;
    if (P.qtab) {  // full covariance: q per component from the table
        v.x = reduce_bits(v.x, vis_q_full(P, f, t, ij_prod(P, i, j), i, false), P.is_int);
        if (!is_auto) v.y = reduce_bits(v.y, vis_q_full(P, f, t, ij_prod(P, i, j), i, true), P.is_int);
        return v;
    }
    const uint32_t row = f * P.n_in;
    const float Ai = __ldg(P.autos + (size_t)(row + i) * P.T + t);
    // autos: s^2 = V_ii^2 / N, q = (2 c A_i) A_i, Im V_ii has no noise and stays;
    // crosses: s^2 = V_ii V_jj / (2N), q = (c A_i) A_j for both components
    const float Aj = is_auto ? Ai : __ldg(P.autos + (size_t)(row + j) * P.T + t);
    const float q = __fmul_rn(__fmul_rn(vis_c(P, f, t, is_auto), Ai), Aj);
    v.x = reduce_bits(v.x, q, P.is_int);
    if (!is_auto) v.y = reduce_bits(v.y, q, P.is_int);
    return v;
}

// Round `ncplx` consecutive complex samples starting at global complex index
// c0, lane k taking samples c0 + k, c0 + k + 32, ...  src and dst may be the
// same (in-place) and may be shared or global memory.
BSG_D void reduce_run(const uint2 *src, uint2 *dst, uint32_t c0, uint32_t ncplx,
                      const VisParams &P, uint32_t lane)
{
    uint32_t c = c0 + lane;
    uint32_t fp = c / P.T;
    uint32_t t = c - fp * P.T;
    uint32_t f = fp / P.P;
    uint32_t p = fp - f * P.P;
    for (uint32_t k = lane; k < ncplx; k += 32) {
        const uint32_t ij = __ldg(P.pairs + p);
        dst[k] = reduce_sample(src[k], ij, f, t, P);
        t += P.rT;
        p += P.qT;
        if (t >= P.T) {
            t -= P.T;
            p++;
        }
        while (p >= P.P) {
            p -= P.P;
            f++;
        }
    }
}

// Same for an even number of samples starting at an even index c0 when the
// time axis is even: each lane takes two consecutive samples (t, t+1) of one
// product per 16-byte access, so the product lookup and the two autos loads
// serve both, and the auto / cross choice is a select (for an auto A_j = A_i,
// the constant is 2c and the imaginary part is kept).
// Round samples (t, t + 1) of product p = (i, j) (ij as in P.pairs) at
// frequency f, held as one 16-byte value.
BSG_D uint4 reduce_pair(uint4 v, uint32_t ij, uint32_t f, uint32_t t, const VisParams &P)
{
    if (P.qtab) {  // full covariance: per-component q from the table
        const uint2 a = reduce_sample(make_uint2(v.x, v.y), ij, f, t, P);
        const uint2 b = reduce_sample(make_uint2(v.z, v.w), ij, f, t + 1, P);
        return make_uint4(a.x, a.y, b.x, b.y);
    }
    const uint32_t i = ij & 0xffffu, j = ij >> 16;
    const uint32_t row = f * P.n_in;
    const float2 Ai = __ldg(reinterpret_cast<const float2 *>(P.autos + (size_t)(row + i) * P.T + t));
    const float2 Aj = __ldg(reinterpret_cast<const float2 *>(P.autos + (size_t)(row + j) * P.T + t));
    const bool is_auto = i == j;
    const float qa = __fmul_rn(__fmul_rn(vis_c(P, f, t, is_auto), Ai.x), Aj.x);
    const float qb = __fmul_rn(__fmul_rn(vis_c(P, f, t + 1, is_auto), Ai.y), Aj.y);
    v.x = reduce_bits(v.x, qa, P.is_int);
    v.z = reduce_bits(v.z, qb, P.is_int);
    if (!is_auto) {
        v.y = reduce_bits(v.y, qa, P.is_int);
        v.w = reduce_bits(v.w, qb, P.is_int);
    }
    return v;
}

BSG_D void reduce_run2(const uint4 *src, uint4 *dst, uint32_t c0, uint32_t ncplx,
                       const VisParams &P, uint32_t lane)
{
    uint32_t c = c0 + 2 * lane;
    uint32_t fp = c / P.T;
    uint32_t t = c - fp * P.T;
    uint32_t f = fp / P.P;
    uint32_t p = fp - f * P.P;
    const uint32_t q64 = 64 / P.T, r64 = 64 % P.T;
    for (uint32_t k = lane; k < ncplx / 2; k += 32) {
        dst[k] = reduce_pair(src[k], __ldg(P.pairs + p), f, t, P);
        t += r64;
        p += q64;
        if (t >= P.T) {
            t -= P.T;
            p++;
        }
        while (p >= P.P) {
            p -= P.P;
            f++;
        }
    }
}

// Precision reduction fused into the 32 x 32 register transpose of a block of
// float32 components (elem size 4), for cubes whose time axis is a multiple
// of 16: a group of 32 floats is 16 consecutive time samples of one product,
// so one product lookup and 16 autos pairs serve the whole group.  Lane k of
// the warp takes groups k, k + 32, ...; its 16-byte chunks are read in a
// lane-rotated order (conflict-free banks) and the autos are loaded in the
// same order; the rotation is undone on the transposed rows.
BSG_D void round_shuffle4_vis(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t c_blk,
                              const VisParams &P, uint32_t lane)
{
    const uint32_t G = Bb / 32;
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t g = lane; g < G; g += 32) {
        const uint8_t *grp = src + 128u * g;
        const uint32_t rot = g & 7u;
        const uint32_t cg = c_blk + 16 * g;       // first sample of the group
        const uint32_t fp = cg / P.T;
        const uint32_t t0 = cg - fp * P.T;
        const uint32_t f = fp / P.P;
        const uint32_t p = fp - f * P.P;
        const uint32_t ij = __ldg(P.pairs + p);
        const uint32_t i = ij & 0xffffu, j = ij >> 16;
        const bool is_auto = i == j;
        const float *ai = P.autos + (size_t)(f * P.n_in + i) * P.T + t0;
        const float *aj = P.autos + (size_t)(f * P.n_in + j) * P.T + t0;
        uint32_t a[32];
        float2 Ai[8], Aj[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t c = (k + rot) & 7u;  // chunk c holds samples t0 + 2c, t0 + 2c + 1
            uint4 v = *reinterpret_cast<const uint4 *>(grp + 16u * c);
            a[4 * k] = v.x;
            a[4 * k + 1] = v.y;
            a[4 * k + 2] = v.z;
            a[4 * k + 3] = v.w;
            Ai[k] = __ldg(reinterpret_cast<const float2 *>(ai + 2 * c));
            Aj[k] = __ldg(reinterpret_cast<const float2 *>(aj + 2 * c));
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const uint32_t t = t0 + 2 * ((k + rot) & 7u);
            const float q0 = __fmul_rn(__fmul_rn(vis_c(P, f, t, is_auto), Ai[k].x), Aj[k].x);
            const float q1 = __fmul_rn(__fmul_rn(vis_c(P, f, t + 1, is_auto), Ai[k].y), Aj[k].y);
            a[4 * k] = reduce_bits(a[4 * k], q0, P.is_int);
            a[4 * k + 2] = reduce_bits(a[4 * k + 2], q1, P.is_int);
            if (!is_auto) {
                a[4 * k + 1] = reduce_bits(a[4 * k + 1], q0, P.is_int);
                a[4 * k + 3] = reduce_bits(a[4 * k + 3], q1, P.is_int);
            }
        }
        // a[m] holds float (m + 4 rot) mod 32 of the group
        transpose32(a);
#pragma unroll
        for (int r = 0; r < 32; r++) d32[r * G + g] = rotl(a[r], 4u * rot);
    }
}

// Round the component (32 bits) at global component index fi (used for the
// verbatim tail).
BSG_D uint32_t reduce_component_at(uint32_t xb, uint64_t fi, const VisParams &P)
{
    uint32_t c = (uint32_t)(fi >> 1);
    uint32_t fp = c / P.T, t = c - fp * P.T;
    uint32_t f = fp / P.P, p = fp - f * P.P;
    uint2 v = (fi & 1) ? make_uint2(0u, xb) : make_uint2(xb, 0u);
    const uint32_t ij = __ldg(P.pairs + p);
    // the imaginary part of an auto is never rounded; everything else as usual
    const uint2 r = reduce_sample(v, ij, f, t, P);
    return (fi & 1) ? r.y : r.x;
}

// ---------------------------------------------------------------------------
// Decoupled look-back over per-block compressed sizes (single-pass output
// placement).  state[t]: 0 = not ready, (1 << 62) | aggregate, (2 << 62) |
// inclusive prefix.  Tiles are taken in order from a counter, so every
// predecessor is held by a running warp; waits are bounded all the same.
// ---------------------------------------------------------------------------
constexpr uint64_t LB_FA = 1ull << 62, LB_FP = 2ull << 62, LB_VM = (1ull << 62) - 1;

// Make a block's compressed size visible to its successors (tile 0 publishes
// its inclusive prefix directly).
BSG_D void lookback_publish(uint64_t *state, uint32_t tile, uint64_t agg, uint32_t lane)
{
    if (lane == 0) st_relaxed_u64(state + tile, (tile == 0 ? LB_FP : LB_FA) | agg);
}

// Exclusive prefix of a block whose size is already published; publishes its
// inclusive prefix.
BSG_D uint64_t lookback_resolve(uint64_t *state, uint32_t tile, uint64_t agg, int *status,
                                uint32_t lane)
{
    constexpr uint64_t FP = LB_FP, VM = LB_VM;
    if (tile == 0) return 0;
    uint64_t excl = 0;
    int64_t base = (int64_t)tile - 1;
    uint32_t spins = 0;
    for (;;) {
        int64_t idx = base - (int64_t)lane;
        uint64_t v = idx >= 0 ? ld_relaxed_u64(state + idx) : FP;
#ifdef BSG_TEST_LOOKBACK_STALL
        // test builds only: predecessors never look ready, so the bounded
        // wait below runs out and reports BSGPU_ERR_TIMEOUT
        if (idx >= 0) v = 0;
#endif
        uint32_t flag = (uint32_t)(v >> 62);
        uint32_t pm = __ballot_sync(FULL, flag == 2);
        uint32_t im = __ballot_sync(FULL, flag == 0);
        uint32_t first = pm ? (uint32_t)(__ffs(pm) - 1) : 31u;
        uint32_t need = first >= 31 ? FULL : ((2u << first) - 1u);
        if (im & need) {
            // predecessors usually publish within a few polls (each poll is a
            // round trip to L2); sleep only once the wait is clearly long
            if (++spins > (1u << 21)) {
                if (lane == 0) set_status(status, BSGPU_ERR_TIMEOUT);
                break;
            }
            if (spins > 4096) __nanosleep(100);
            continue;
        }
        uint64_t x = lane <= first ? (v & VM) : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
        excl += x;
        if (pm) break;
        base -= 32;
    }
    if (lane == 0) st_relaxed_u64(state + tile, FP | (excl + agg));
    return excl;
}

BSG_D uint64_t lookback(uint64_t *state, uint32_t tile, uint64_t agg, int *status,
                        uint32_t lane)
{
    lookback_publish(state, tile, agg, lane);
    return lookback_resolve(state, tile, agg, status, lane);
}

// ---------------------------------------------------------------------------
// Compress: [round ->] bitshuffle -> LZ4 -> placed by look-back
// ---------------------------------------------------------------------------
// Round (for a cube) and bit-transpose block `tile` from `in` into `tmp`.
BSG_D void compress_prepare(const CodecArgs &a, uint32_t tile, uint8_t *in, uint8_t *tmp,
                            uint32_t lane)
{
    const uint32_t Bb = block_elems_of(a, tile);
    // the block starts at a whole complex sample (B is a multiple of 8)
    const uint32_t c0 = (uint32_t)(((uint64_t)tile * a.B * a.es) >> 3);
    const uint32_t ncplx = Bb * a.es / 8;
    if (a.vis.enabled && !a.vis.qtab && a.es == 4 && Bb % 32u == 0 && a.vis.T % 16u == 0) {
        round_shuffle4_vis(in, tmp, Bb, c0, a.vis, lane);
        return;
    }
    if (a.vis.enabled) {
        if ((a.vis.T & 1u) == 0) {  // c0 and ncplx are even
            uint4 *b4 = reinterpret_cast<uint4 *>(in);
            reduce_run2(b4, b4, c0, ncplx, a.vis, lane);
        } else {
            uint2 *b2 = reinterpret_cast<uint2 *>(in);
            reduce_run(b2, b2, c0, ncplx, a.vis, lane);
        }
        __syncwarp();
    }
    shuffle_block(in, tmp, Bb, a.es, lane);
}

// Write block `tile` (its 4-byte length field and cs LZ4 bytes at `blk`, in
// shared or global memory) at stream offset D, with the index entry, the
// chunk header (block 0) and, after the last block, the verbatim tail.
BSG_D void compress_place(const CodecArgs &a, uint32_t tile, const uint8_t *blk, uint32_t cs,
                          uint64_t D, uint32_t lane)
{
    if (D + 4 + cs > a.out_cap) {
        if (lane == 0) set_status(a.status, BSGPU_ERR_SPACE);
        return;
    }
    copy_out(blk, a.out + D, 4 + cs, lane);
    if (a.block_offsets && lane == 0) a.block_offsets[tile] = D;
    if (tile == 0) write_chunk_header(a.out, a.n_elem * a.es, a.B * a.es, lane);
    if (tile + 1 == a.nb) {
        // the (n mod 8) trailing elements follow the last block verbatim
        const uint64_t end = D + 4 + cs;
        const uint64_t first = a.n_elem - a.tail_elems;
        const uint32_t tb = a.tail_elems * a.es;
        if (end + tb > a.out_cap) {
            if (lane == 0) set_status(a.status, BSGPU_ERR_SPACE);
            return;
        }
        if (a.vis.enabled) {
            // the tail as 32-bit components, each rounded like any other
            const uint32_t tc = tb / 4;
            const uint64_t c0 = first * a.es / 4;
            if (lane < tc) {
                const uint32_t *src = reinterpret_cast<const uint32_t *>(a.in);
                const uint64_t fi = c0 + lane;
                const uint32_t x = src[2 * vis_src(a.vis, fi >> 1) + (fi & 1)];
                const uint32_t u = reduce_component_at(x, fi, a.vis);
                for (int k = 0; k < 4; k++) a.out[end + 4 * lane + k] = (uint8_t)(u >> (8 * k));
            }
        } else {
            for (uint32_t k = lane; k < tb; k += 32) a.out[end + k] = a.in[first * a.es + k];
        }
        if (lane == 0) *a.out_bytes = end + tb;
    }
}

// Drop the L2 lines of a placed block's staging slot without writing them
// back: the slot is dead until the warp encodes into it again, and without
// this the streaming traffic evicts the dirty slot lines to DRAM for
// nothing (measured on a 64-chunk batch: the compress launch's DRAM writes
// 611 -> 393 MB for a 231 MB stream, 1008 -> 960 us).  The single-stream
// fast kernel does not use it: its slots stay in L2 (its DRAM writes match
// its stream) and the extra instructions cost it 2 %.  Only lines wholly inside [p, p + bytes) go (the lines at the
// ends may hold a neighbouring slot); the caller has synchronised the warp
// after its reads of the slot.
BSG_D void discard_slot(const uint8_t *p, uint32_t bytes, uint32_t lane)
{
    const uintptr_t a0 = ((uintptr_t)p + 127u) & ~(uintptr_t)127u;
    const uintptr_t a1 = ((uintptr_t)p + bytes) & ~(uintptr_t)127u;
    for (uintptr_t x = a0 + 128u * lane; x < a1; x += 128u * 32u)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(x) : "memory");
}

// LZ4-encode the bit-rows in `tmp` into `dst` after a 4-byte length field;
// returns the LZ4 size.
template <int LEVEL, int HBITS>
BSG_D uint32_t compress_encode(const CodecArgs &a, uint32_t Bb, const uint8_t *tmp, uint8_t *dst,
                               void *scratch, uint32_t lane)
{
    const uint32_t S = Bb * a.es;
    // bit-rows are Bb/8 bytes long: the previous row is one of the candidates
    uint32_t cs = LEVEL >= 1
        ? lz4_encode_warp<1, HBITS>(tmp, S, Bb / 8, dst + 4, static_cast<uint16_t *>(scratch))
        : lz4_encode_bitmap(tmp, S, Bb / 8, dst + 4, static_cast<uint32_t *>(scratch));
    if (cs == 0xffffffffu) {  // progress guard (not reachable for valid sizes)
        if (lane == 0) set_status(a.status, BSGPU_ERR_CUDA);
        cs = 0;
    }
    if (lane == 0) put_be32(dst, cs);
    __syncwarp();
    return cs;
}

// Place block `ptile`, staged in global `slot` (4 + cs bytes): the bytes come
// back into the warp's block buffer `buf` (free until the next block's load,
// with the encoder's scratch after it) by one bulk copy that runs while the
// look-back finds the block's offset, and go out from there.
BSG_D void place_staged(const CodecArgs &a, uint32_t ptile, const uint8_t *slot, uint32_t cs,
                        uint8_t *buf, uint64_t *bar, uint32_t &parity, uint32_t lane)
{
    const uint32_t bytes = r16(4 + cs);
    fence_proxy_async_all();  // the slot was written by this warp's generic stores
    __syncwarp();
    if (lane == 0) {
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(buf, slot, bytes, bar);
    }
    const uint64_t excl = lookback_resolve(a.tile_state, ptile, 4ull + cs, a.status, lane);
    if (!mbar_wait_bounded(bar, parity) && lane == 0) set_status(a.status, BSGPU_ERR_TIMEOUT);
    parity ^= 1u;
    compress_place(a, ptile, buf, cs, 12 + excl, lane);
}

// LZ4-encode the bit-rows in `tmp` into `out`, place the block by look-back
// and write it.
template <uint32_t MAXB, int LEVEL>
BSG_D void compress_finish(const CodecArgs &a, uint32_t tile, uint8_t *tmp, uint8_t *out,
                           void *scratch, uint32_t lane)
{
    using L = CompPlan<MAXB, LEVEL>;
    const uint32_t Bb = block_elems_of(a, tile);
    const uint32_t cs = compress_encode<LEVEL, L::HBITS>(a, Bb, tmp, out, scratch, lane);
    const uint64_t excl = lookback(a.tile_state, tile, 4ull + cs, a.status, lane);
    compress_place(a, tile, out, cs, 12 + excl, lane);
}

// ---------------------------------------------------------------------------
// Compress, fast path: blocks of at most 8 KiB of 4- or 8-byte elements
// ---------------------------------------------------------------------------
template <int LEVEL>
struct FastPlan {
    static constexpr uint32_t MAXB = 8192;
    static constexpr uint32_t TMP = r16(MAXB + 16);  // staged block, then its bit-rows
    static constexpr int HBITS = 11;
    // level 1: the hash table; level 0: the fast encoder's bitmaps and tables
    static constexpr uint32_t SCR = LEVEL >= 1 ? (2u << HBITS) : LZ4_FAST_SCRATCH;
    static constexpr uint32_t BYTES = TMP + r16(SCR) + 16;
};

static_assert(FAST_SLOT_BYTES >= r16(4 + lz4b(8192) + 32), "staging slot too small");

// Round the 32 components of one group (16 samples t0 .. t0 + 15 of one
// product) held as a[m] = component (m + 4 rot) mod 32.  GEN: int32 data or a
// per-sample compensated c; otherwise float32 with the constant c, which is
// kept as its own instantiation so that the common case carries no per-value
// selects.
template <bool GEN>
BSG_D void round_group(const VisParams &P, uint32_t (&a)[32], uint32_t rot, uint32_t f,
                       uint32_t t0, const float *ai, const float *aj, bool is_auto)
{
    if (GEN) {
        // c per sample: the compensated table (two adjacent samples per
        // 8-byte load) or the constant; the data type is one branch per group
        const float *crow = P.cft ? P.cft + (size_t)f * P.T + t0 : nullptr;
        const float mul = is_auto ? 2.0f : 1.0f;  // exact: c2 = 2 c
        auto qs = [&](uint32_t c, float &q0, float &q1) {
            const float2 Ai = __ldg(reinterpret_cast<const float2 *>(ai + 2 * c));
            const float2 Aj = __ldg(reinterpret_cast<const float2 *>(aj + 2 * c));
            const float2 cc = crow ? __ldg(reinterpret_cast<const float2 *>(crow + 2 * c))
                                   : make_float2(P.c, P.c);
            q0 = __fmul_rn(__fmul_rn(__fmul_rn(cc.x, mul), Ai.x), Aj.x);
            q1 = __fmul_rn(__fmul_rn(__fmul_rn(cc.y, mul), Ai.y), Aj.y);
        };
        if (P.is_int) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                float q0, q1;
                qs((k + rot) & 7u, q0, q1);
                a[4 * k] = reduce_bits(a[4 * k], q0, true);
                a[4 * k + 2] = reduce_bits(a[4 * k + 2], q1, true);
                if (!is_auto) {
                    a[4 * k + 1] = reduce_bits(a[4 * k + 1], q0, true);
                    a[4 * k + 3] = reduce_bits(a[4 * k + 3], q1, true);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                float q0, q1;
                qs((k + rot) & 7u, q0, q1);
                a[4 * k] = __float_as_uint(reduce_one(__uint_as_float(a[4 * k]), q0));
                a[4 * k + 2] = __float_as_uint(reduce_one(__uint_as_float(a[4 * k + 2]), q1));
                if (!is_auto) {
                    a[4 * k + 1] = __float_as_uint(reduce_one(__uint_as_float(a[4 * k + 1]), q0));
                    a[4 * k + 3] = __float_as_uint(reduce_one(__uint_as_float(a[4 * k + 3]), q1));
                }
            }
        }
        return;
    }
    const float cc = is_auto ? P.c2 : P.c;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const uint32_t c = (k + rot) & 7u;  // chunk c: samples t0 + 2c, t0 + 2c + 1
        const float2 Ai = __ldg(reinterpret_cast<const float2 *>(ai + 2 * c));
        const float2 Aj = __ldg(reinterpret_cast<const float2 *>(aj + 2 * c));
        const float q0 = __fmul_rn(__fmul_rn(cc, Ai.x), Aj.x);
        const float q1 = __fmul_rn(__fmul_rn(cc, Ai.y), Aj.y);
        a[4 * k] = __float_as_uint(reduce_one(__uint_as_float(a[4 * k]), q0));
        a[4 * k + 2] = __float_as_uint(reduce_one(__uint_as_float(a[4 * k + 2]), q1));
        if (!is_auto) {
            a[4 * k + 1] = __float_as_uint(reduce_one(__uint_as_float(a[4 * k + 1]), q0));
            a[4 * k + 3] = __float_as_uint(reduce_one(__uint_as_float(a[4 * k + 3]), q1));
        }
    }
}

// Precision reduction of one group of 32 components (16 consecutive time
// samples of one product, the time axis being a multiple of 16) held in
// registers in lane-rotated chunk order: a[m] is component (m + 4 (g & 7)) mod 32.
// With the full-covariance table, each component has its own q (the Re and
// Im rows of the product at the group's 16 times).
BSG_D void round_group_full(const VisParams &P, uint32_t (&a)[32], uint32_t rot, const float *qre,
                            const float *qim, bool is_auto)
{
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const uint32_t c = (k + rot) & 7u;   // chunk c: samples t0 + 2c, t0 + 2c + 1
        const float2 qr = __ldg(reinterpret_cast<const float2 *>(qre + 2 * c));
        const float2 qi = __ldg(reinterpret_cast<const float2 *>(qim + 2 * c));
        a[4 * k] = reduce_bits(a[4 * k], qr.x, P.is_int);
        a[4 * k + 2] = reduce_bits(a[4 * k + 2], qr.y, P.is_int);
        if (!is_auto) {   // the imaginary part of an auto stays
            a[4 * k + 1] = reduce_bits(a[4 * k + 1], qi.x, P.is_int);
            a[4 * k + 3] = reduce_bits(a[4 * k + 3], qi.y, P.is_int);
        }
    }
}

template <bool GEN>
struct VisGroupRound {
    const VisParams *P;
    uint32_t c_blk;  // complex index of the block's first sample
    BSG_D void operator()(uint32_t g, uint32_t (&a)[32]) const
    {
        const uint32_t rot = g & 7u;
        const uint32_t cg = c_blk + 16 * g;
        const uint32_t fp = fastdiv(cg, P->dT);
        const uint32_t t0 = cg - fp * P->T;
        const uint32_t f = fastdiv(fp, P->dP);
        const uint32_t p = fp - f * P->P;
        const uint32_t ij = __ldg(P->pairs + p);
        const uint32_t i = ij & 0xffffu, j = ij >> 16;
        const bool is_auto = i == j;
        if (GEN && P->qtab) {
            // full covariance: the q rows of the Re and Im components ([F][M][T])
            const float *qre = P->qtab + ((size_t)f * P->M + p) * P->T + t0;
            const float *qim = P->qtab + ((size_t)f * P->M + P->P + p - i - 1) * P->T + t0;
            round_group_full(*P, a, rot, qre, is_auto ? qre : qim, is_auto);
            return;
        }
        const float *ai = P->autos + (size_t)(f * P->n_in + i) * P->T + t0;
        const float *aj = P->autos + (size_t)(f * P->n_in + j) * P->T + t0;
        round_group<GEN>(*P, a, rot, f, t0, ai, aj, is_auto);
    }
};

struct NoRound {
    BSG_D void operator()(uint32_t, uint32_t (&)[32]) const {}
};

// ---------------------------------------------------------------------------
// Decompress: LZ4 decode -> bit un-transpose, every block at once
// ---------------------------------------------------------------------------

// One shared buffer for in-place decoding of blocks of at most 8 KiB: the
// block's compressed image at its end, the output from its start (see
// decompress_inplace_kernel for the margin).  Placement (an image of at most
// 4 + lz4b(8192) bytes, 32 before the end, 16 for the phase) and in-place
// safety (image start - (S - clen) >= 72).
constexpr uint32_t INPLACE_BUF = 8352;

// The same buffer for any block size up to maxb (decompress_inplace_any_kernel):
// room for the image (4 + lz4b(maxb), placed at most 48 bytes before the end)
// and the in-place margin (at least S + 2 S / 255 + 49 bytes).
__host__ __device__ constexpr uint32_t inplace_any_buf(uint32_t maxb)
{
    return maxb <= 8192 ? INPLACE_BUF : r16(maxb + 2u * maxb / 255u + 160u);
}
static_assert(inplace_any_buf(16384) >= 4 + lz4b(16384) + 48 &&
                  inplace_any_buf(16384) >= 16384 + 2 * 16384 / 255 + 49 &&
                  inplace_any_buf(65536) >= 4 + lz4b(65536) + 48 &&
                  inplace_any_buf(65536) >= 65536 + 2 * 65536 / 255 + 49 &&
                  INPLACE_BUF >= 4 + lz4b(8192) + 48 && INPLACE_BUF >= 8192 + 2 * 8192 / 255 + 49,
              "in-place buffer");
static_assert(INPLACE_BUF >= 4 + lz4b(8192) + 48, "in-place buffer: image does not fit");
static_assert(INPLACE_BUF >= 8192 + 119, "in-place buffer: margin below the LZ4 bound");

struct DecLoad {
    bool bulk;       // a bulk copy is in flight on the barrier
    bool ok;         // offsets passed the range checks
    uint32_t delta;  // shared index of the first stream byte (D & 15)
    uint32_t clen;   // LZ4 bytes of the block
    uint32_t eidx;   // shared index this lane's edge byte goes to (or ~0)
    uint8_t ebyte;
    uint32_t off;    // where in the buffer the block's image starts (see dec_issue)
};

// Bytes [D, Dn) of the stream go to shared index x - (D & ~15) of the image
// (dst + r.off): the 16-byte aligned middle by one bulk copy, the ragged head
// and tail (< 16 bytes each) by plain loads held in registers until the block
// is processed.  end_bytes = 0 puts the image at dst; otherwise at the end of
// a buffer of end_bytes bytes (a 16-byte boundary at least 32 bytes before
// its end), for decoding in place (decompress_inplace_kernel).
BSG_D DecLoad dec_issue(const CodecArgs &a, uint32_t tile, uint8_t *dst, uint64_t *bar,
                        uint32_t lane, uint32_t end_bytes = 0)
{
    DecLoad r;
    r.bulk = false;
    r.ok = false;
    r.eidx = ~0u;
    r.ebyte = 0;
    r.delta = 0;
    r.clen = 0;
    r.off = 0;
    const uint32_t Bb = block_elems_of(a, tile);
    const uint64_t tail_b = (uint64_t)a.tail_elems * a.es;
    if (a.in_bytes < 12 + tail_b) return r;
    const uint64_t D = a.block_offsets[tile];
    const uint64_t Dn = tile + 1 < a.nb ? a.block_offsets[tile + 1] : a.in_bytes - tail_b;
    if (D < 12 || Dn < D + 4 || Dn > a.in_bytes || Dn - D - 4 > lz4b(Bb * a.es)) return r;
    r.ok = true;
    r.clen = (uint32_t)(Dn - D - 4);
    if (end_bytes) {
        // the range check above bounds Dn - D by 4 + lz4b(S) <= end_bytes - 48
        r.off = (end_bytes - (uint32_t)(Dn - D) - 32u) & ~15u;
        dst += r.off;
    }
    // alignment is a property of the absolute address, not of the offset
    const uint64_t g0 = (uint64_t)(uintptr_t)(a.in + D), gn = g0 + (Dn - D);
    const uint64_t base = g0 & ~15ull;
    r.delta = (uint32_t)(g0 - base);
    const uint64_t A0 = (g0 + 15) & ~15ull, A1 = gn & ~15ull;
    const uint64_t head_end = A0 < gn ? A0 : gn;
    const uint64_t tail_beg = A1 > A0 ? A1 : A0;
    if (A1 > A0) {
        if (lane == 0) {
            mbar_arrive_expect_tx(bar, (uint32_t)(A1 - A0));
            bulk_g2s(dst + (A0 - base), reinterpret_cast<const void *>(A0), (uint32_t)(A1 - A0),
                     bar);
        }
        r.bulk = true;
    }
    uint64_t x = lane < 16 ? g0 + lane : tail_beg + (lane - 16);
    if ((lane < 16 && x < head_end) || (lane >= 16 && x < gn)) {
        r.ebyte = *reinterpret_cast<const uint8_t *>(x);
        r.eidx = (uint32_t)(x - base);
    }
    return r;
}


// ---------------------------------------------------------------------------
// Block index of a stream that carries none: the chain of 4-byte big-endian
// length fields (reading R11) walked from offset 12.  The walk is serial
// (each block starts where the previous one ends), so its speed is the
// latency of one read per block; read from global memory that is a DRAM
// round trip per block.  Instead the stream's bytes stream through shared
// memory in windows of WALK_WIN bytes, WALK_NBUF of them in flight on the
// bulk-copy engine, and lane 0 walks the windows.  The ragged first and last
// (< 16) bytes of the stream, which no bulk copy can move, are read once by
// the warp beforehand.  Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr uint32_t WALK_WIN = 16384, WALK_NBUF = 8;
constexpr uint32_t WALK_SMEM = WALK_WIN * WALK_NBUF + 8 * WALK_NBUF + 32;

struct ChainWalk {
    uintptr_t in, a0, a1;   // stream start; its 16-byte aligned middle [a0, a1)
    uint32_t nwin;          // windows over [a0, a1)
    uint8_t *buf;           // WALK_NBUF windows
    uint64_t *bar;          // one barrier per window buffer
    uint8_t *edge;          // bytes [in, a0) at edge[0..15], [a1, end) at edge[16..31]
    bool ok;                // every wait ended in time
};

BSG_D void walk_issue(ChainWalk &w, uint32_t k)
{
    const uintptr_t lo = w.a0 + (uintptr_t)k * WALK_WIN;
    const uintptr_t hi = lo + WALK_WIN < w.a1 ? lo + WALK_WIN : w.a1;
    uint64_t *bar = w.bar + k % WALK_NBUF;
    mbar_arrive_expect_tx(bar, (uint32_t)(hi - lo));
    bulk_g2s(w.buf + (size_t)(k % WALK_NBUF) * WALK_WIN, reinterpret_cast<const void *>(lo),
             (uint32_t)(hi - lo), bar);
}

// Byte at address x of the stream; window k (that holds x) must have arrived.
BSG_D uint32_t walk_byte(const ChainWalk &w, uintptr_t x)
{
    if (x < w.a0) return w.edge[x - w.in];
    if (x >= w.a1) return w.edge[16 + (x - w.a1)];
    const uintptr_t r = x - w.a0;
    return w.buf[(size_t)((r / WALK_WIN) % WALK_NBUF) * WALK_WIN + r % WALK_WIN];
}

// Lane 0: block offsets of blocks 0 .. nb-1 of the stream `in` (in_bytes
// long, tail_b verbatim bytes at its end) into offsets[]; false when the
// chain does not end exactly at the verbatim tail.  The other lanes only
// help with the edge bytes.
BSG_D bool chain_walk_staged(const uint8_t *in, uint64_t in_bytes, uint32_t nb, uint64_t tail_b,
                             uint64_t *offsets, uint8_t *smem, uint32_t lane, bool &timely)
{
    ChainWalk w;
    w.in = (uintptr_t)in;
    const uintptr_t end = w.in + in_bytes;
    w.a0 = (w.in + 15) & ~(uintptr_t)15;
    w.a1 = end & ~(uintptr_t)15;
    if (w.a1 < w.a0) w.a1 = w.a0;   // a stream shorter than one aligned chunk
    w.nwin = (uint32_t)((w.a1 - w.a0 + WALK_WIN - 1) / WALK_WIN);
    w.buf = smem;
    w.bar = reinterpret_cast<uint64_t *>(smem + (size_t)WALK_WIN * WALK_NBUF);
    w.edge = reinterpret_cast<uint8_t *>(w.bar + WALK_NBUF);
    w.ok = true;
    // the ragged edges: [in, a0) and [a1, end) (each under 16 bytes; when the
    // stream has no aligned middle, [in, end) is split between the two)
    if (lane < 16 && w.in + lane < (w.a0 < end ? w.a0 : end)) w.edge[lane] = in[lane];
    if (lane >= 16 && w.a1 + (lane - 16) < end && w.a1 + (lane - 16) >= w.a0)
        w.edge[lane] = *reinterpret_cast<const uint8_t *>(w.a1 + (lane - 16));
    if (lane == 0)
        for (uint32_t k = 0; k < WALK_NBUF; k++) mbar_init(w.bar + k, 1);
    fence_mbar_init();
    __syncwarp();
    bool good = true;
    if (lane == 0) {
        // windows are issued, waited for and released in order: window k
        // reuses the buffer of window k - WALK_NBUF once that one has been
        // waited for and lies wholly before the next length field
        int32_t issued = 0, done = 0;
        const int32_t nwin = (int32_t)w.nwin;
        while (issued < nwin && issued < (int32_t)WALK_NBUF) walk_issue(w, (uint32_t)issued++);
        uint64_t D = 12;
        uint32_t b = 0;
        for (; b < nb; b++) {
            if (D + 4 > in_bytes) {
                good = false;
                break;
            }
            offsets[b] = D;
            const uintptr_t x = w.in + D;
            // windows holding the part of x .. x+3 inside [a0, a1)
            const uintptr_t lo = x > w.a0 ? x : w.a0, hi = x + 3 < w.a1 ? x + 3 : w.a1 - 1;
            if (lo <= hi && w.a1 > w.a0) {
                const int32_t wb = (int32_t)((hi - w.a0) / WALK_WIN);
                while (done <= wb && w.ok) {
                    if (done >= issued) {        // skipped ahead: its buffer is free
                        fence_proxy_async_smem();
                        walk_issue(w, (uint32_t)issued++);
                    }
                    if (!mbar_wait_bounded(w.bar + done % WALK_NBUF, (uint32_t)(done / WALK_NBUF) & 1u))
                        w.ok = false;
                    done++;
                }
            }
            if (!w.ok) {
                good = false;
                break;
            }
            const uint32_t len = (walk_byte(w, x) << 24) | (walk_byte(w, x + 1) << 16) |
                                 (walk_byte(w, x + 2) << 8) | walk_byte(w, x + 3);
            D += 4ull + len;
            // prefetch: windows whose buffers held waited-for windows wholly
            // before the next length field
            const uintptr_t nx = w.in + (D < in_bytes ? D : in_bytes);
            const int32_t nwa = nx < w.a0 ? 0 : (int32_t)((nx - w.a0) / WALK_WIN);
            while (issued < nwin && issued - (int32_t)WALK_NBUF < done &&
                   issued - (int32_t)WALK_NBUF < nwa) {
                fence_proxy_async_smem();   // the reads of the buffer before its next bulk write
                walk_issue(w, (uint32_t)issued++);
            }
        }
        for (; b < nb; b++) offsets[b] = in_bytes;   // fails the decoder's range check
        good = good && D + tail_b == in_bytes;
        // no bulk copy may still be writing when the warp moves on
        while (done < issued) {
            if (!mbar_wait_bounded(w.bar + done % WALK_NBUF, (uint32_t)(done / WALK_NBUF) & 1u))
                w.ok = false;
            done++;
        }
    }
    timely = __shfl_sync(FULL, w.ok ? 1u : 0u, 0) != 0;
    return __shfl_sync(FULL, good ? 1u : 0u, 0) != 0;
}

// ---------------------------------------------------------------------------
// The same block index recovered in parallel, exactly.  The stream's block
// area [12, end) is cut into K segments, each at least SEG_M + 1 of the
// largest blocks long.  Warp k takes as its start the first position of its
// segment that reads as a block start (a length field in [1, lz4b(S)] whose
// chain stays inside the area for SEG_DEPTH more blocks, or ends exactly at
// its end) and walks the chain: it counts the blocks that start in the
// segment and records the first SEG_M of them and the first SEG_M chain
// positions past the segment.  Warp 0 starts at 12, so its walk is the true
// chain.  A false start of warp k either dies (and the check below fails)
// or falls onto the true chain; the chains meet where warp k - 1's positions
// past its segment (true, by induction) meet warp k's first positions, and
// from there warp k walks the true chain.  A scan checks that every pair
// meets within SEG_M steps, corrects each count by the meeting point,
// checks that the counts add up to nb and the last walk ends at the area's
// end, and numbers the blocks; only then are the offsets written.  A stream
// that fails any check takes the staged serial walk instead, so the index
// is exact either way.
// ---------------------------------------------------------------------------
constexpr uint32_t SEG_MAX = 2048;   // segments (warps) of the parallel recovery
constexpr uint32_t SEG_M = 8;        // chain positions recorded at each end of a segment
constexpr uint32_t SEG_DEPTH = 8;    // blocks a start candidate's chain must survive

struct SegRec {
    uint64_t head[SEG_M];    // the first chain positions inside the segment (from the start)
    uint64_t after[SEG_M];   // the first chain positions at or past the segment's end
    uint64_t start, base;    // after the scan: the true first block start, its block number
    uint32_t c, nh;          // blocks counted inside the segment; entries of head
    uint32_t na, ok;         // entries of after; the walk stayed valid
};
static_assert(sizeof(SegRec) == 2 * 8 * SEG_M + 32, "segment record");
constexpr size_t SEG_WS_REC = 256 + sizeof(SegRec) * SEG_MAX;

// Big-endian 32-bit length field at offset p of the stream (4 byte loads,
// issued together).
BSG_D uint32_t stream_be32(const uint8_t *in, uint64_t p)
{
    const uint32_t b0 = __ldg(in + p), b1 = __ldg(in + p + 1), b2 = __ldg(in + p + 2),
                   b3 = __ldg(in + p + 3);
    return (b0 << 24) | (b1 << 16) | (b2 << 8) | b3;
}

// Whether offset p reads as a block start: a length field in [1, maxlen]
// and a chain that stays inside [12, end) for `depth` more blocks or ends
// exactly at end.
BSG_D bool seg_plausible(const uint8_t *in, uint64_t p, uint64_t end, uint32_t maxlen,
                         uint32_t depth)
{
    for (uint32_t v = 0; v <= depth; v++) {
        if (p == end) return true;
        if (p + 4 > end) return false;
        const uint32_t len = stream_be32(in, p);
        if (len < 1 || len > maxlen || p + 4 + len > end) return false;
        p += 4ull + len;
    }
    return true;
}

template <typename K>
inline cudaError_t launch_warp_kernel(K kernel, uint32_t smem, uint32_t grid, cudaStream_t s,
                                      const CodecArgs &a)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, 32, smem, s>>>(a);
    return cudaGetLastError();
}


}  // namespace bsg
