// bsgpu kernels for sm_103a: precision reduction (Sec. 3.2), Bitshuffle
// (Sec. 4.2) and per-block LZ4 with framing (Sec. 4.1, 4.2.1), and the
// inverse path.  One warp per CTA; each warp owns one block (the unit the
// paper threads over, Sec. 4.2.1) at a time, staged in shared memory by the
// bulk-copy (TMA) engine with the next block prefetched.
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

uint32_t compress_smem_bytes(uint32_t maxb, int level)
{
    if (level >= 1)
        return maxb <= 8192 ? CompPlan<8192, 1>::BYTES
                            : (maxb <= 16384 ? CompPlan<16384, 1>::BYTES : CompPlan<65536, 1>::BYTES);
    return maxb <= 8192 ? CompPlan<8192, 0>::BYTES
                        : (maxb <= 16384 ? CompPlan<16384, 0>::BYTES : CompPlan<65536, 0>::BYTES);
}
uint32_t decompress_smem_bytes(uint32_t maxb)
{
    return maxb <= 8192 ? DecPlan<8192>::BYTES
                        : (maxb <= 16384 ? DecPlan<16384>::BYTES : DecPlan<65536>::BYTES);
}
uint32_t shuffle_smem_bytes(uint32_t maxb)
{
    return maxb <= 8192 ? ShufPlan<8192>::BYTES
                        : (maxb <= 16384 ? ShufPlan<16384>::BYTES : ShufPlan<65536>::BYTES);
}

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
// Round one complex sample (re, im bits) of product p = (i, j) at (f, t).
BSG_D uint2 reduce_sample(uint2 v, uint32_t ij, uint32_t f, uint32_t t, const VisParams &P)
{
    const uint32_t i = ij & 0xffffu, j = ij >> 16;
    const uint32_t row = f * P.n_in;
    const float Ai = __ldg(P.autos + (size_t)(row + i) * P.T + t);
    const bool is_auto = i == j;
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
        const uint32_t ij = __ldg(P.pairs + p);
        const uint32_t i = ij & 0xffffu, j = ij >> 16;
        const uint32_t row = f * P.n_in;
        const float2 Ai = __ldg(reinterpret_cast<const float2 *>(P.autos + (size_t)(row + i) * P.T + t));
        const float2 Aj = __ldg(reinterpret_cast<const float2 *>(P.autos + (size_t)(row + j) * P.T + t));
        const bool is_auto = i == j;
        const float qa = __fmul_rn(__fmul_rn(vis_c(P, f, t, is_auto), Ai.x), Aj.x);
        const float qb = __fmul_rn(__fmul_rn(vis_c(P, f, t + 1, is_auto), Ai.y), Aj.y);
        uint4 v = src[k];
        v.x = reduce_bits(v.x, qa, P.is_int);
        v.z = reduce_bits(v.z, qb, P.is_int);
        if (!is_auto) {
            v.y = reduce_bits(v.y, qa, P.is_int);
            v.w = reduce_bits(v.w, qb, P.is_int);
        }
        dst[k] = v;
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

// Tables for the rounding: autos[f][i][t] = Re V(f, (i,i), t) and
// pairs[p] = i | j << 16 for the upper-triangle product order.
__global__ void vis_tables_kernel(const float *__restrict__ vis, float *__restrict__ autos,
                                  uint32_t *__restrict__ pairs, uint32_t n_freq, uint32_t n_in,
                                  uint32_t T, int is_int)
{
    const uint32_t P = n_in * (n_in + 1) / 2;
    const uint64_t n_auto = (uint64_t)n_freq * n_in * T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_auto; x += stride) {
        uint32_t t = (uint32_t)(x % T);
        uint64_t fi = x / T;
        uint32_t i = (uint32_t)(fi % n_in);
        uint64_t f = fi / n_in;
        uint64_t pii = (uint64_t)i * n_in - (uint64_t)i * (i - 1) / 2;
        const size_t at = ((f * P + pii) * T + t) * 2;
        // int32 autos are converted to float32 (round to nearest)
        autos[x] = is_int ? __int2float_rn(reinterpret_cast<const int32_t *>(vis)[at]) : vis[at];
    }
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
        // row i holds products [i n - i (i-1)/2, (i+1) n - (i+1) i / 2)
        uint32_t lo = 0, hi = n_in - 1;
        while (lo < hi) {
            uint32_t mid = (lo + hi + 1) / 2;
            uint64_t start = (uint64_t)mid * n_in - (uint64_t)mid * (mid - 1) / 2;
            if (start <= p) lo = mid; else hi = mid - 1;
        }
        uint64_t start = (uint64_t)lo * n_in - (uint64_t)lo * (lo - 1) / 2;
        uint32_t j = lo + (uint32_t)(p - start);
        pairs[p] = lo | (j << 16);
    }
}

// Sec. 3.2's compensation: per (freq, time) sample, c is recomputed from
// f m with m = min over cross products of 1 - |V_ij|^2 / (V_ii V_jj) in
// float32 (each operation rounded to nearest; a negative or NaN value counts
// as 0; no cross product gives 1), c = fl32(6 (f m) / N) in fp64.  One CTA per
// (frequency, chunk of up to 1024 time samples); the minimum of non-negative
// floats is taken on their bit patterns.
__global__ void __launch_bounds__(256) vis_compensation_kernel(const void *__restrict__ vis,
                                                               VisParams P, float *cft,
                                                               uint32_t n_freq, double f,
                                                               double N)
{
    __shared__ uint32_t mins[1024];
    const uint32_t nchunk = (P.T + 1023) / 1024;
    for (uint32_t cb = blockIdx.x; cb < n_freq * nchunk; cb += gridDim.x) {
        const uint32_t fr = cb / nchunk, t0 = (cb % nchunk) * 1024;
        const uint32_t tn = P.T - t0 < 1024 ? P.T - t0 : 1024;
        for (uint32_t t = threadIdx.x; t < tn; t += blockDim.x) mins[t] = __float_as_uint(1.0f);
        __syncthreads();
        for (uint64_t e = threadIdx.x; e < (uint64_t)P.P * tn; e += blockDim.x) {
            const uint32_t p = (uint32_t)(e / tn), t = t0 + (uint32_t)(e % tn);
            const uint32_t ij = __ldg(P.pairs + p);
            const uint32_t i = ij & 0xffffu, j = ij >> 16;
            if (i == j) continue;
            const float Ai = __ldg(P.autos + ((size_t)fr * P.n_in + i) * P.T + t);
            const float Aj = __ldg(P.autos + ((size_t)fr * P.n_in + j) * P.T + t);
            const size_t at = (((size_t)fr * P.P + p) * P.T + t) * 2;
            float re, im;
            if (P.is_int) {
                re = __int2float_rn(reinterpret_cast<const int32_t *>(vis)[at]);
                im = __int2float_rn(reinterpret_cast<const int32_t *>(vis)[at + 1]);
            } else {
                re = reinterpret_cast<const float *>(vis)[at];
                im = reinterpret_cast<const float *>(vis)[at + 1];
            }
            const float num = __fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im));
            const float den = __fmul_rn(Ai, Aj);
            float om = __fsub_rn(1.0f, __fdiv_rn(num, den));
            if (!(om >= 0.0f)) om = 0.0f;
            atomicMin(&mins[t - t0], __float_as_uint(om));
        }
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < tn; t += blockDim.x) {
            const double fe = __dmul_rn(f, (double)__uint_as_float(mins[t]));
            cft[(size_t)fr * P.T + t0 + t] = __double2float_rn(__ddiv_rn(__dmul_rn(6.0, fe), N));
        }
        __syncthreads();
    }
}

// Standalone precision reduction: each warp rounds runs of 1024 samples.
__global__ void __launch_bounds__(256) reduce_precision_kernel(const uint2 *__restrict__ in,
                                                               uint2 *__restrict__ out,
                                                               uint64_t n_cplx, VisParams P)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    constexpr uint32_t RUN = 1024;
    for (uint64_t r = warp * RUN; r < n_cplx; r += nwarps * RUN) {
        uint32_t cnt = (uint32_t)(n_cplx - r < RUN ? n_cplx - r : RUN);
        if ((P.T & 1u) == 0)  // r is even and so is cnt (n_cplx = F P T is even)
            reduce_run2(reinterpret_cast<const uint4 *>(in + r), reinterpret_cast<uint4 *>(out + r),
                        (uint32_t)r, cnt, P, lane);
        else
            reduce_run(in + r, out + r, (uint32_t)r, cnt, P, lane);
    }
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
    if (a.vis.enabled && a.es == 4 && Bb % 32u == 0 && a.vis.T % 16u == 0) {
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
                const uint32_t u = reduce_component_at(src[c0 + lane], c0 + lane, a.vis);
                for (int k = 0; k < 4; k++) a.out[end + 4 * lane + k] = (uint8_t)(u >> (8 * k));
            }
        } else {
            for (uint32_t k = lane; k < tb; k += 32) a.out[end + k] = a.in[first * a.es + k];
        }
        if (lane == 0) *a.out_bytes = end + tb;
    }
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

// One warp per CTA, persistent.  Per block: wait for its bulk copy into `in`,
// round + transpose into `tmp`, start the next block's copy into `in`, then
// LZ4 into `out`, look-back placement and the write-out, which overlap the
// next block's copy.
template <uint32_t MAXB, int LEVEL>
__global__ void __launch_bounds__(32, MAXB <= 8192 ? 9 : 1)
    compress_kernel(const __grid_constant__ CodecArgs a)
{
    using L = CompPlan<MAXB, LEVEL>;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *in = sm;
    uint8_t *tmp = sm + L::IN;
    uint8_t *out = tmp + L::TMP;
    void *scratch = out + L::OUT;
    uint64_t *bar = reinterpret_cast<uint64_t *>(out + L::OUT + r16(L::SCR));
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;
    uint32_t tile = a.tile_begin + grab_tile(a.tile_counter, lane);
    bool pend = tile < a.tile_end && load_block(in, a.in + (uint64_t)tile * a.B * a.es,
                                                block_elems_of(a, tile) * a.es, bar, lane);
    while (tile < a.tile_end) {
        if (pend) {
            if (!mbar_wait_bounded(bar, parity) && lane == 0) set_status(a.status, BSGPU_ERR_TIMEOUT);
            parity ^= 1u;
        }
        compress_prepare(a, tile, in, tmp, lane);
        __syncwarp();
        const uint32_t nxt = a.tile_begin + grab_tile(a.tile_counter, lane);
        pend = false;
        if (nxt < a.tile_end) {
            // the transpose's reads of `in` (generic proxy) precede the async write
            fence_proxy_async_smem();
            __syncwarp();
            pend = load_block(in, a.in + (uint64_t)nxt * a.B * a.es, block_elems_of(a, nxt) * a.es,
                              bar, lane);
        }
        compress_finish<MAXB, LEVEL>(a, tile, tmp, out, scratch, lane);
        __syncwarp();
        tile = nxt;
    }
}

// ---------------------------------------------------------------------------
// Compress, fast path: blocks of at most 8 KiB of 4- or 8-byte elements
// ---------------------------------------------------------------------------
template <int LEVEL>
struct FastPlan {
    static constexpr uint32_t MAXB = 8192;
    static constexpr uint32_t TMP = r16(MAXB + 16);  // staged block, then its bit-rows
    static constexpr int HBITS = 11;
    static constexpr uint32_t SCR = LEVEL >= 1 ? (2u << HBITS) : 2u * 4u * (MAXB / 128u + 2u);
    static constexpr uint32_t BYTES = TMP + r16(SCR) + 16;
};

uint32_t compress_fast_smem_bytes(int level)
{
    return level >= 1 ? FastPlan<1>::BYTES : FastPlan<0>::BYTES;
}

template <int LEVEL, int ES, bool GEN = false>
__global__ void compress_fast_kernel(const __grid_constant__ CodecArgs a);

uint32_t compress_fast_blocks_per_sm(int level, uint32_t es)
{
    int n = 0;
    const uint32_t smem = compress_fast_smem_bytes(level);
    cudaError_t e;
    if (es == 8)
        e = level >= 1
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<1, 8>, 32, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<0, 8>, 32, smem);
    else
        e = level >= 1
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<1, 4>, 32, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<0, 4>, 32, smem);
    return e == cudaSuccess && n > 0 ? (uint32_t)n : 1u;
}

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
    const float cc = is_auto ? P.c2 : P.c;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const uint32_t c = (k + rot) & 7u;  // chunk c: samples t0 + 2c, t0 + 2c + 1
        const float2 Ai = __ldg(reinterpret_cast<const float2 *>(ai + 2 * c));
        const float2 Aj = __ldg(reinterpret_cast<const float2 *>(aj + 2 * c));
        if (GEN) {
            const float q0 = __fmul_rn(__fmul_rn(vis_c(P, f, t0 + 2 * c, is_auto), Ai.x), Aj.x);
            const float q1 = __fmul_rn(__fmul_rn(vis_c(P, f, t0 + 2 * c + 1, is_auto), Ai.y), Aj.y);
            a[4 * k] = reduce_bits(a[4 * k], q0, P.is_int);
            a[4 * k + 2] = reduce_bits(a[4 * k + 2], q1, P.is_int);
            if (!is_auto) {
                a[4 * k + 1] = reduce_bits(a[4 * k + 1], q0, P.is_int);
                a[4 * k + 3] = reduce_bits(a[4 * k + 3], q1, P.is_int);
            }
        } else {
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
}

// Precision reduction of one group of 32 components (16 consecutive time
// samples of one product, the time axis being a multiple of 16) held in
// registers in lane-rotated chunk order: a[m] is component (m + 4 (g & 7)) mod 32.
template <bool GEN>
struct VisGroupRound {
    const VisParams *P;
    uint32_t c_blk;  // complex index of the block's first sample
    BSG_D void operator()(uint32_t g, uint32_t (&a)[32]) const
    {
        const uint32_t rot = g & 7u;
        const uint32_t cg = c_blk + 16 * g;
        const uint32_t fp = cg / P->T;
        const uint32_t t0 = cg - fp * P->T;
        const uint32_t f = fp / P->P;
        const uint32_t p = fp - f * P->P;
        const uint32_t ij = __ldg(P->pairs + p);
        const uint32_t i = ij & 0xffffu, j = ij >> 16;
        const bool is_auto = i == j;
        const float *ai = P->autos + (size_t)(f * P->n_in + i) * P->T + t0;
        const float *aj = P->autos + (size_t)(f * P->n_in + j) * P->T + t0;
        round_group<GEN>(*P, a, rot, f, t0, ai, aj, is_auto);
    }
};

struct NoRound {
    BSG_D void operator()(uint32_t, uint32_t (&)[32]) const {}
};

// One warp per CTA, persistent, one shared buffer: bulk-copy the block in,
// round + bit-transpose it in place through registers, LZ4-encode it into
// this warp's staging slot in global memory (it stays in L2), publish its
// size, and place the PREVIOUS block: by then its predecessors have long
// published theirs, so the look-back rarely waits.  GEN (4-byte elements of a
// cube only): int32 components or a compensated c (see round_group).
template <int LEVEL, int ES, bool GEN>
__global__ void __launch_bounds__(32, 16) compress_fast_kernel(const __grid_constant__ CodecArgs a)
{
    using L = FastPlan<LEVEL>;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *tmp = sm;
    void *scratch = sm + L::TMP;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::TMP + r16(L::SCR));
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint8_t *slot0 = a.slots + (size_t)(2 * blockIdx.x) * FAST_SLOT_BYTES;
    uint8_t *slot1 = slot0 + FAST_SLOT_BYTES;
    uint32_t parity = 0;
    uint32_t ptile = ~0u, pcs = 0;  // the block waiting to be placed, in slot1
    uint32_t tile = grab_tile(a.tile_counter, lane);
    while (tile < a.tile_end) {
        const uint32_t Bb = a.B;  // the fast path takes full blocks only
        if (load_block(tmp, a.in + (uint64_t)tile * a.B * a.es, Bb * a.es, bar, lane)) {
            if (!mbar_wait_bounded(bar, parity) && lane == 0) set_status(a.status, BSGPU_ERR_TIMEOUT);
            parity ^= 1u;
        }
        if (ES == 8) {
            if (a.vis.enabled) {
                // one complex sample per element: round them in place first
                const uint32_t c0 = (uint32_t)((uint64_t)tile * a.B);
                if ((a.vis.T & 1u) == 0) {
                    uint4 *b4 = reinterpret_cast<uint4 *>(tmp);
                    reduce_run2(b4, b4, c0, Bb, a.vis, lane);
                } else {
                    uint2 *b2 = reinterpret_cast<uint2 *>(tmp);
                    reduce_run(b2, b2, c0, Bb, a.vis, lane);
                }
                __syncwarp();
            }
            shuffle8_inplace(tmp, Bb, lane);
        } else if (a.vis.enabled) {
            shuffle4_inplace(tmp, Bb, lane,
                             VisGroupRound<GEN>{&a.vis, (uint32_t)(((uint64_t)tile * a.B) >> 1)});
        } else {
            shuffle4_inplace(tmp, Bb, lane, NoRound{});
        }
        __syncwarp();
        uint32_t cs;
        if (LEVEL == 0 && (Bb * ES) % 128u == 0) {
            cs = lz4_encode_bitmap_fast(tmp, Bb * ES, Bb / 8, slot0 + 4);
            if (lane == 0) put_be32(slot0, cs);
            __syncwarp();
        } else {
            cs = compress_encode<LEVEL, L::HBITS>(a, Bb, tmp, slot0, scratch, lane);
        }
        lookback_publish(a.tile_state, tile, 4ull + cs, lane);
        const uint32_t nxt = grab_tile(a.tile_counter, lane);
        if (ptile != ~0u) {
            const uint64_t excl = lookback_resolve(a.tile_state, ptile, 4ull + pcs, a.status, lane);
            compress_place(a, ptile, slot1, pcs, 12 + excl, lane);
        }
        __syncwarp();
        ptile = tile;
        pcs = cs;
        uint8_t *t = slot0;
        slot0 = slot1;
        slot1 = t;
        tile = nxt;
        // the next load overwrites `tmp`: the async proxy follows the generic reads
        fence_proxy_async_smem();
        __syncwarp();
    }
    if (ptile != ~0u) {
        const uint64_t excl = lookback_resolve(a.tile_state, ptile, 4ull + pcs, a.status, lane);
        compress_place(a, ptile, slot1, pcs, 12 + excl, lane);
    }
}

// n_elem < 8: no block; header plus the elements verbatim (rounded for a cube).
__global__ void compress_small_kernel(const __grid_constant__ CodecArgs a)
{
    const uint32_t lane = threadIdx.x & 31u;
    write_chunk_header(a.out, a.n_elem * a.es, a.B * a.es, lane);
    const uint32_t tb = a.tail_elems * a.es;
    if (a.vis.enabled) {
        if (lane < tb / 4) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(a.in);
            const uint32_t u = reduce_component_at(src[lane], lane, a.vis);
            for (int k = 0; k < 4; k++) a.out[12 + 4 * lane + k] = (uint8_t)(u >> (8 * k));
        }
    } else {
        for (uint32_t k = lane; k < tb; k += 32) a.out[12 + k] = a.in[k];
    }
    if (lane == 0) *a.out_bytes = 12 + tb;
}

// ---------------------------------------------------------------------------
// Decompress: LZ4 decode -> bit un-transpose, every block at once
// ---------------------------------------------------------------------------

struct DecLoad {
    bool bulk;       // a bulk copy is in flight on the barrier
    bool ok;         // offsets passed the range checks
    uint32_t delta;  // shared index of the first stream byte (D & 15)
    uint32_t clen;   // LZ4 bytes of the block
    uint32_t eidx;   // shared index this lane's edge byte goes to (or ~0)
    uint8_t ebyte;
};

// Bytes [D, Dn) of the stream go to shared index x - (D & ~15): the 16-byte
// aligned middle by one bulk copy, the ragged head and tail (< 16 bytes each)
// by plain loads held in registers until the block is processed.
BSG_D DecLoad dec_issue(const CodecArgs &a, uint32_t tile, uint8_t *dst, uint64_t *bar,
                        uint32_t lane)
{
    DecLoad r;
    r.bulk = false;
    r.ok = false;
    r.eidx = ~0u;
    r.ebyte = 0;
    r.delta = 0;
    r.clen = 0;
    const uint32_t Bb = block_elems_of(a, tile);
    const uint64_t tail_b = (uint64_t)a.tail_elems * a.es;
    if (a.in_bytes < 12 + tail_b) return r;
    const uint64_t D = a.block_offsets[tile];
    const uint64_t Dn = tile + 1 < a.nb ? a.block_offsets[tile + 1] : a.in_bytes - tail_b;
    if (D < 12 || Dn < D + 4 || Dn > a.in_bytes || Dn - D - 4 > lz4b(Bb * a.es)) return r;
    r.ok = true;
    r.clen = (uint32_t)(Dn - D - 4);
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

// One warp per CTA, persistent.  Per block: wait for its stream bytes in
// `comp`, LZ4-decode into `dec`, start the next block's copy into `comp`,
// un-transpose `dec` in place and bulk-store it (blocks the register paths
// cannot take are un-transposed into `comp` and stored before the next copy).
// ES: 4 or 8 compiles the in-place register un-transpose for that element
// size; 0 compiles only the general path.
template <uint32_t MAXB, int ES>
__global__ void __launch_bounds__(32, MAXB <= 8192 ? 13 : 1)
    decompress_kernel(const __grid_constant__ CodecArgs a)
{
    using L = DecPlan<MAXB>;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *comp = sm;
    uint8_t *dec = sm + L::COMP;
    uint64_t *bar = reinterpret_cast<uint64_t *>(dec + L::DEC);
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;
    bool header_checked = false;
    uint32_t tile = grab_tile(a.tile_counter, lane);
    DecLoad ld;
    if (tile < a.nb) ld = dec_issue(a, tile, comp, bar, lane);
    while (tile < a.nb) {
        const DecLoad cur = ld;
        if (cur.bulk) {
            if (!mbar_wait_bounded(bar, parity) && lane == 0) set_status(a.status, BSGPU_ERR_TIMEOUT);
            parity ^= 1u;
        }
        if (!header_checked) {
            header_checked = true;
            uint32_t ok = 1;
            if (lane < 12) {
                uint8_t want = lane < 8 ? (uint8_t)((a.n_elem * a.es) >> (8 * (7 - lane)))
                                        : (uint8_t)(((uint64_t)a.B * a.es) >> (8 * (11 - lane)));
                ok = a.in_bytes >= 12 && a.in[lane] == want;
            }
            if (__ballot_sync(FULL, !ok) && lane == 0) set_status(a.status, BSGPU_ERR_CORRUPT);
        }
        const uint32_t Bb = block_elems_of(a, tile);
        const uint32_t S = Bb * a.es;
        const uint32_t nxt = grab_tile(a.tile_counter, lane);
        // the previous block's bulk store must have finished reading `dec`
        if (lane == 0) bulk_wait_read0();
        __syncwarp();
        bool good = cur.ok;
        if (good) {
            if (cur.eidx != ~0u) comp[cur.eidx] = cur.ebyte;
            __syncwarp();
            good = get_be32(comp + cur.delta) == cur.clen &&
                   lz4_decode_warp(comp, cur.delta + 4, cur.clen, dec, S) == 0;
        }
        if (!good && lane == 0) set_status(a.status, BSGPU_ERR_CORRUPT);
        uint8_t *dst = a.out + (uint64_t)tile * a.B * a.es;
        const bool inplace = ES != 0 && MAXB <= 8192 && unshuffle_inplace_ok(a.es, Bb);
        if (good && !inplace) {
            unshuffle_block(dec, comp, Bb, a.es, lane);
            __syncwarp();
            for (uint32_t k = lane; k < S; k += 32) dst[k] = comp[k];
        }
        __syncwarp();
        ld.bulk = false;
        ld.ok = false;
        if (nxt < a.nb) {
            // `comp` was last read by the generic proxy
            fence_proxy_async_smem();
            __syncwarp();
            ld = dec_issue(a, nxt, comp, bar, lane);
        }
        if (good && inplace) {
            if (ES == 4)
                unshuffle4_inplace(dec, Bb, lane);
            else if (ES == 8)
                unshuffle8_inplace(dec, Bb, lane);
            __syncwarp();
            if ((S & 15u) == 0 && ((uintptr_t)dst & 15u) == 0) {
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    bulk_s2g(dst, dec, S);
                    bulk_commit();
                }
            } else {
                for (uint32_t k = lane; k < S; k += 32) dst[k] = dec[k];
            }
        }
        if (tile + 1 == a.nb) {
            const uint32_t tb = a.tail_elems * a.es;
            const uint64_t first = (a.n_elem - a.tail_elems) * a.es;
            if (a.in_bytes >= tb)
                for (uint32_t k = lane; k < tb; k += 32)
                    a.out[first + k] = a.in[a.in_bytes - tb + k];
        }
        __syncwarp();
        tile = nxt;
    }
    if (lane == 0) bulk_wait0();
    __syncwarp();
}

// Block offsets by walking the chain of 4-byte length fields (one thread).
__global__ void chain_walk_kernel(const __grid_constant__ CodecArgs a, uint64_t *offsets)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t tail_b = (uint64_t)a.tail_elems * a.es;
    uint64_t D = 12;
    uint32_t b = 0;
    bool bad = false;
    for (; b < a.nb; b++) {
        if (D + 4 > a.in_bytes) {
            bad = true;
            break;
        }
        offsets[b] = D;
        D += 4 + (uint64_t)get_be32(a.in + D);
    }
    for (; b < a.nb; b++) offsets[b] = a.in_bytes;  // fails the range check
    if (bad || D + tail_b != a.in_bytes) set_status(a.status, BSGPU_ERR_CORRUPT);
}

// n_elem < 8: the elements sit verbatim after the header.
__global__ void decompress_small_kernel(const __grid_constant__ CodecArgs a)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t tb = a.tail_elems * a.es;
    bool ok = a.in_bytes == 12ull + tb;
    if (ok && lane < 12) {
        uint8_t want = lane < 8 ? (uint8_t)((a.n_elem * a.es) >> (8 * (7 - lane)))
                                : (uint8_t)(((uint64_t)a.B * a.es) >> (8 * (11 - lane)));
        ok = a.in[lane] == want;
    }
    if (__ballot_sync(FULL, !ok)) {
        if (lane == 0) set_status(a.status, BSGPU_ERR_CORRUPT);
        return;
    }
    for (uint32_t k = lane; k < tb; k += 32) a.out[k] = a.in[12 + k];
}

// ---------------------------------------------------------------------------
// Standalone Bitshuffle / un-Bitshuffle (no LZ4): static tiles per warp
// ---------------------------------------------------------------------------
template <uint32_t MAXB, bool INV>
__global__ void __launch_bounds__(32) shuffle_kernel(const __grid_constant__ CodecArgs a)
{
    using L = ShufPlan<MAXB>;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *buf[2] = {sm, sm + L::BUF};
    uint8_t *ob = sm + 2 * L::BUF;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ob + L::BUF);
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (a.nb == 0) {  // fewer than 8 elements: plain copy
        if (blockIdx.x == 0)
            for (uint32_t k = lane; k < a.n_elem * a.es; k += 32) a.out[k] = a.in[k];
        return;
    }
    uint32_t parity[2] = {0u, 0u};
    bool pend[2] = {false, false};
    uint32_t tile = blockIdx.x;
    int cur = 0;
    if (tile < a.nb)
        pend[0] = load_block(buf[0], a.in + (uint64_t)tile * a.B * a.es,
                             block_elems_of(a, tile) * a.es, &bar[0], lane);
    while (tile < a.nb) {
        const uint32_t nxt = tile + gridDim.x;
        if (pend[cur]) {
            if (!mbar_wait_bounded(&bar[cur], parity[cur]) && lane == 0)
                set_status(a.status, BSGPU_ERR_TIMEOUT);
            parity[cur] ^= 1u;
            pend[cur] = false;
        }
        if (nxt < a.nb) {
            fence_proxy_async_smem();
            __syncwarp();
            pend[cur ^ 1] = load_block(buf[cur ^ 1], a.in + (uint64_t)nxt * a.B * a.es,
                                       block_elems_of(a, nxt) * a.es, &bar[cur ^ 1], lane);
        }
        const uint32_t Bb = block_elems_of(a, tile);
        const uint32_t S = Bb * a.es;
        // the previous bulk store from `ob` must have finished reading it
        if (lane == 0) bulk_wait_read0();
        __syncwarp();
        if (INV)
            unshuffle_block(buf[cur], ob, Bb, a.es, lane);
        else
            shuffle_block(buf[cur], ob, Bb, a.es, lane);
        __syncwarp();
        uint8_t *dst = a.out + (uint64_t)tile * a.B * a.es;
        if ((S & 15u) == 0 && ((uintptr_t)dst & 15u) == 0) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                bulk_s2g(dst, ob, S);
                bulk_commit();
            }
        } else {
            for (uint32_t k = lane; k < S; k += 32) dst[k] = ob[k];
        }
        if (tile + 1 == a.nb) {
            const uint64_t first = (a.n_elem - a.tail_elems) * a.es;
            for (uint32_t k = lane; k < a.tail_elems * a.es; k += 32)
                a.out[first + k] = a.in[first + k];
        }
        __syncwarp();
        tile = nxt;
        cur ^= 1;
    }
    if (lane == 0) bulk_wait0();
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t launch_warp_kernel(K kernel, uint32_t smem, uint32_t grid, cudaStream_t s,
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

cudaError_t launch_vis_compensation(const void *vis, const VisParams &P, uint32_t n_freq,
                                    double f, double N, cudaStream_t s)
{
    const uint64_t work = (uint64_t)n_freq * ((P.T + 1023) / 1024);
    const uint32_t grid = (uint32_t)(work < 8192 ? work : 8192);
    vis_compensation_kernel<<<grid ? grid : 1, 256, 0, s>>>(vis, P, const_cast<float *>(P.cft),
                                                            n_freq, f, N);
    return cudaGetLastError();
}

cudaError_t launch_vis_tables(const float *vis, float *autos, uint32_t *pairs, uint32_t n_freq,
                              uint32_t n_in, uint32_t T, int is_int, cudaStream_t s)
{
    uint64_t n = (uint64_t)n_freq * n_in * T;
    uint64_t P = (uint64_t)n_in * (n_in + 1) / 2;
    uint64_t work = n > P ? n : P;
    uint32_t blocks = (uint32_t)((work + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks == 0) blocks = 1;
    vis_tables_kernel<<<blocks, 256, 0, s>>>(vis, autos, pairs, n_freq, n_in, T, is_int);
    return cudaGetLastError();
}

cudaError_t launch_reduce_precision(const float *in, float *out, uint64_t n_cplx,
                                    const VisParams &v, uint32_t grid, cudaStream_t s)
{
    reduce_precision_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const uint2 *>(in),
                                                 reinterpret_cast<uint2 *>(out), n_cplx, v);
    return cudaGetLastError();
}

cudaError_t launch_shuffle(const CodecArgs &a, bool inverse, uint32_t maxb, uint32_t grid,
                           cudaStream_t s)
{
    uint32_t smem = shuffle_smem_bytes(maxb);
    if (maxb <= 8192)
        return inverse ? launch_warp_kernel(shuffle_kernel<8192, true>, smem, grid, s, a)
                       : launch_warp_kernel(shuffle_kernel<8192, false>, smem, grid, s, a);
    if (maxb <= 16384)
        return inverse ? launch_warp_kernel(shuffle_kernel<16384, true>, smem, grid, s, a)
                       : launch_warp_kernel(shuffle_kernel<16384, false>, smem, grid, s, a);
    return inverse ? launch_warp_kernel(shuffle_kernel<65536, true>, smem, grid, s, a)
                   : launch_warp_kernel(shuffle_kernel<65536, false>, smem, grid, s, a);
}

cudaError_t launch_compress(const CodecArgs &a, uint32_t maxb, uint32_t grid, cudaStream_t s)
{
    uint32_t smem = compress_smem_bytes(maxb, a.level);
    if (a.level >= 1) {
        if (maxb <= 8192) return launch_warp_kernel(compress_kernel<8192, 1>, smem, grid, s, a);
        if (maxb <= 16384) return launch_warp_kernel(compress_kernel<16384, 1>, smem, grid, s, a);
        return launch_warp_kernel(compress_kernel<65536, 1>, smem, grid, s, a);
    }
    if (maxb <= 8192) return launch_warp_kernel(compress_kernel<8192, 0>, smem, grid, s, a);
    if (maxb <= 16384) return launch_warp_kernel(compress_kernel<16384, 0>, smem, grid, s, a);
    return launch_warp_kernel(compress_kernel<65536, 0>, smem, grid, s, a);
}

cudaError_t launch_compress_fast(const CodecArgs &a, uint32_t grid, cudaStream_t s)
{
    const uint32_t smem = compress_fast_smem_bytes(a.level);
    if (a.es == 8)
        return a.level >= 1 ? launch_warp_kernel(compress_fast_kernel<1, 8>, smem, grid, s, a)
                            : launch_warp_kernel(compress_fast_kernel<0, 8>, smem, grid, s, a);
    if (a.vis.enabled && (a.vis.is_int || a.vis.cft))
        return a.level >= 1 ? launch_warp_kernel(compress_fast_kernel<1, 4, true>, smem, grid, s, a)
                            : launch_warp_kernel(compress_fast_kernel<0, 4, true>, smem, grid, s, a);
    return a.level >= 1 ? launch_warp_kernel(compress_fast_kernel<1, 4>, smem, grid, s, a)
                        : launch_warp_kernel(compress_fast_kernel<0, 4>, smem, grid, s, a);
}

cudaError_t launch_compress_small(const CodecArgs &a, cudaStream_t s)
{
    compress_small_kernel<<<1, 32, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_decompress(const CodecArgs &a, uint32_t maxb, uint32_t grid, cudaStream_t s)
{
    if (a.nb == 0) {
        decompress_small_kernel<<<1, 32, 0, s>>>(a);
        return cudaGetLastError();
    }
    uint32_t smem = decompress_smem_bytes(maxb);
    if (maxb <= 8192) {
        if (a.es == 4) return launch_warp_kernel(decompress_kernel<8192, 4>, smem, grid, s, a);
        if (a.es == 8) return launch_warp_kernel(decompress_kernel<8192, 8>, smem, grid, s, a);
        return launch_warp_kernel(decompress_kernel<8192, 0>, smem, grid, s, a);
    }
    if (maxb <= 16384) return launch_warp_kernel(decompress_kernel<16384, 0>, smem, grid, s, a);
    return launch_warp_kernel(decompress_kernel<65536, 0>, smem, grid, s, a);
}

cudaError_t launch_chain_walk(const CodecArgs &a, uint64_t *offsets, cudaStream_t s)
{
    chain_walk_kernel<<<1, 32, 0, s>>>(a, offsets);
    return cudaGetLastError();
}

}  // namespace bsg
