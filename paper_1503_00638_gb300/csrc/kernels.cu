// bsgpu kernels for sm_103a: precision reduction (Sec. 3.2), Bitshuffle
// (Sec. 4.2) and per-block LZ4 with framing (Sec. 4.1, 4.2.1), and the
// inverse path.  One warp per CTA; each warp owns one block (the unit the
// paper threads over, Sec. 4.2.1) at a time, staged in shared memory by the
// bulk-copy (TMA) engine with the next block prefetched.
#include <cuda_runtime.h>

#include "compress_fast.cuh"

namespace bsg {

template <uint32_t MAXB, int LEVEL>
constexpr uint32_t comp_plan_bytes(bool staged)
{
    return staged ? CompPlan<MAXB, LEVEL>::BYTES_STAGED : CompPlan<MAXB, LEVEL>::BYTES;
}
uint32_t compress_smem_bytes(uint32_t maxb, int level, bool staged)
{
    if (level >= 1)
        return maxb <= 8192 ? comp_plan_bytes<8192, 1>(staged)
             : maxb <= 16384 ? comp_plan_bytes<16384, 1>(staged)
             : maxb <= 32768 ? comp_plan_bytes<32768, 1>(staged) : comp_plan_bytes<65536, 1>(staged);
    return maxb <= 8192 ? comp_plan_bytes<8192, 0>(staged)
         : maxb <= 16384 ? comp_plan_bytes<16384, 0>(staged)
         : maxb <= 32768 ? comp_plan_bytes<32768, 0>(staged) : comp_plan_bytes<65536, 0>(staged);
}
uint32_t compress_slot_bytes(uint32_t maxb)
{
    return maxb <= 8192 ? CompPlan<8192, 0>::SLOT
         : maxb <= 16384 ? CompPlan<16384, 0>::SLOT
         : maxb <= 32768 ? CompPlan<32768, 0>::SLOT : CompPlan<65536, 0>::SLOT;
}
uint32_t decompress_smem_bytes(uint32_t maxb)
{
    return maxb <= 8192 ? DecPlan<8192>::BYTES
         : maxb <= 16384 ? DecPlan<16384>::BYTES
         : maxb <= 32768 ? DecPlan<32768>::BYTES : DecPlan<65536>::BYTES;
}
uint32_t shuffle_smem_bytes(uint32_t maxb)
{
    // (blocks over 16 KiB share the largest plan)
    return maxb <= 8192 ? ShufPlan<8192>::BYTES
                        : (maxb <= 16384 ? ShufPlan<16384>::BYTES : ShufPlan<65536>::BYTES);
}

// Tables for the rounding: autos[f][i][t] = Re V(f, (i,i), t) and
// pairs[p] = i | j << 16 for the upper-triangle product order.
__global__ void vis_tables_kernel(const float *__restrict__ vis, VisParams V, uint32_t n_freq)
{
    float *autos = const_cast<float *>(V.autos);
    uint32_t *pairs = const_cast<uint32_t *>(V.pairs);
    const uint32_t n_in = V.n_in, T = V.T;
    const int is_int = V.is_int;
    const uint32_t P = n_in * (n_in + 1) / 2;
    const uint64_t n_auto = (uint64_t)n_freq * n_in * T;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_auto; x += stride) {
        uint32_t t = (uint32_t)(x % T);
        uint64_t fi = x / T;
        uint32_t i = (uint32_t)(fi % n_in);
        uint64_t f = fi / n_in;
        uint64_t pii = (uint64_t)i * n_in - (uint64_t)i * (i - 1) / 2;
        const size_t at = vis_src(V, (f * P + pii) * T + t) * 2;
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
// floats is taken on their bit patterns (order-free, so per-thread minima
// merged by one atomic each give the same result as any other order).
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
        if (!P.tslow && tn <= blockDim.x) {
            // time-fastest cube: thread (p0, tl) takes time t0 + tl of products
            // p0, p0 + per, ... (the lanes of a product read consecutive
            // samples), keeps its minimum in a register and merges it once
            const uint32_t per = blockDim.x / tn, tl = threadIdx.x % tn, p0 = threadIdx.x / tn;
            if (p0 < per) {
                const uint32_t t = t0 + tl;
                const float *arow = P.autos + (size_t)fr * P.n_in * P.T + t;
                uint32_t m = __float_as_uint(1.0f);
                // eight samples (and their product entries) are loaded before
                // any is used, with no branch between the loads, so that they
                // are in flight together
                const uint2 *vrow = reinterpret_cast<const uint2 *>(vis) + (size_t)fr * P.P * P.T + t;
                for (uint32_t pb = p0; pb < P.P; pb += 8 * per) {
                    uint2 v[8];
                    uint32_t ijs[8];
#pragma unroll
                    for (uint32_t k = 0; k < 8; k++) {
                        const uint32_t p = pb + k * per;
                        const bool in = p < P.P;
                        v[k] = in ? __ldg(vrow + (size_t)p * P.T) : make_uint2(0u, 0u);
                        ijs[k] = in ? __ldg(P.pairs + p) : 0u;   // 0: the auto (0, 0), skipped
                    }
#pragma unroll
                    for (uint32_t k = 0; k < 8; k++) {
                        const uint32_t i = ijs[k] & 0xffffu, j = ijs[k] >> 16;
                        if (i == j) continue;
                        const float Ai = __ldg(arow + (size_t)i * P.T);
                        const float Aj = __ldg(arow + (size_t)j * P.T);
                        float re, im;
                        if (P.is_int) {
                            re = __int2float_rn((int32_t)v[k].x);
                            im = __int2float_rn((int32_t)v[k].y);
                        } else {
                            re = __uint_as_float(v[k].x);
                            im = __uint_as_float(v[k].y);
                        }
                        const float num = __fadd_rn(__fmul_rn(re, re), __fmul_rn(im, im));
                        const float den = __fmul_rn(Ai, Aj);
                        float om = __fsub_rn(1.0f, __fdiv_rn(num, den));
                        if (!(om >= 0.0f)) om = 0.0f;
                        m = min(m, __float_as_uint(om));
                    }
                }
                atomicMin(&mins[tl], m);
            }
        } else
        for (uint64_t e = threadIdx.x; e < (uint64_t)P.P * tn; e += blockDim.x) {
            const uint32_t p = (uint32_t)(e / tn), t = t0 + (uint32_t)(e % tn);
            const uint32_t ij = __ldg(P.pairs + p);
            const uint32_t i = ij & 0xffffu, j = ij >> 16;
            if (i == j) continue;
            const float Ai = __ldg(P.autos + ((size_t)fr * P.n_in + i) * P.T + t);
            const float Aj = __ldg(P.autos + ((size_t)fr * P.n_in + j) * P.T + t);
            const size_t at = vis_src(P, ((size_t)fr * P.P + p) * P.T + t) * 2;
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

// Sec. 3.1's full covariance for small arrays (Eq. rad_full1-3) and the noise
// of Eq. noise, s^2 = 1 / (C^-1)_kk, for every component of every (freq,
// time) sample; q = fl32(12 f s^2) goes to P.qtab (0: not rounded).
//
// C is the covariance of the real components (Re V_ij for i <= j, Im V_ij
// for i < j) of the correlation matrix of circular complex Gaussian signals:
// C_ab = tr(D_a V D_b V) / N, with D_a the Hermitian matrix for which
// tr(D_a X) is component a of X.  Let E_b be the dual basis (X = sum_b
// x_b E_b, so tr(D_a E_b) = delta_ab and sum_b D_b tr(E_b Y) = Y for every
// Hermitian Y) and W = V^-1.  Then H_bc = N tr(E_b W E_c W) gives
// (C H)_ac = sum_b tr(D_a V D_b V) tr(E_b W E_c W) = tr(D_a V (W E_c W) V)
// = tr(D_a E_c) = delta_ac: C^-1 = H, whose diagonal is
//   N W_ii^2                        for Re V_ii,
//   2 N (W_ii W_jj + Re(W_ij^2))    for Re V_ij (i < j),
//   2 N (W_ii W_jj - Re(W_ij^2))    for Im V_ij (i < j).
// So the n x n complex inverse (O(n^3) in fp64) replaces the n^2 x n^2 real
// one (O(n^6)).  C is positive definite exactly when V is definite (V or -V
// positive definite: H is quadratic in W); otherwise the sample stays
// unrounded.
//
// One thread per sample, 32 samples per CTA (persistent): the sample's lower
// triangles sit in shared memory as [element][lane] (the lanes of one
// element in consecutive words: no bank conflicts), so every lane of every
// fp64 instruction works (on GB300 fp64 issues at a small fraction of the
// fp32 rate, and a warp instruction costs the same whatever its lanes).
// Per sample: V's lower triangle; Cholesky V = L L^H in place (of -V when
// V_00 < 0); X = L^-1 in place, column by column (for column j, every L
// entry still needed lies right of it or below the current row); W = X^H X
// for the diagonal and for each product.  The q table is [F][M][T], so the
// lanes' writes (consecutive times) coalesce.
__device__ __forceinline__ uint32_t tri_el(uint32_t r, uint32_t c) { return r * (r + 1) / 2 + c; }

__global__ void __launch_bounds__(32) full_noise_kernel(const void *__restrict__ vis, VisParams P,
                                                        uint32_t n_freq, double f, double N,
                                                        double *s2_out)
{
    extern __shared__ double fsm[];
    const uint32_t lane = threadIdx.x;
    const uint32_t n = P.n_in, NP = P.P, M = P.M;   // NP = n (n + 1) / 2 triangle elements
    double *Ar = fsm + lane, *Ai = fsm + 32 * NP + lane, *D = fsm + 64 * NP + lane;
    float *qtab = const_cast<float *>(P.qtab);
    const uint64_t n_smp = (uint64_t)n_freq * P.T;
    for (uint64_t base = (uint64_t)blockIdx.x * 32; base < n_smp; base += (uint64_t)gridDim.x * 32) {
        const uint64_t smp = base + lane;
        const bool live = smp < n_smp;
        const uint32_t fr = live ? (uint32_t)(smp / P.T) : 0u, t = live ? (uint32_t)(smp % P.T) : 0u;
        bool ok = live;
        if (live) {
            for (uint32_t p = 0; p < NP; p++) {
                const uint32_t ij = __ldg(P.pairs + p), i = ij & 0xffffu, j = ij >> 16;
                const size_t at = vis_src(P, ((size_t)fr * NP + p) * P.T + t) * 2;
                double re, im;   // the stored values (int32 through float32)
                if (P.is_int) {
                    re = (double)(float)__ldg(reinterpret_cast<const int32_t *>(vis) + at);
                    im = (double)(float)__ldg(reinterpret_cast<const int32_t *>(vis) + at + 1);
                } else {
                    re = __ldg(reinterpret_cast<const float *>(vis) + at);
                    im = __ldg(reinterpret_cast<const float *>(vis) + at + 1);
                }
                Ar[32 * tri_el(j, i)] = re;   // V_ji = conj(V_ij)
                Ai[32 * tri_el(j, i)] = -im;
            }
            const double sg = Ar[0] < 0.0 ? -1.0 : 1.0;
            for (uint32_t j = 0; j < n; j++) {
                double d = sg * Ar[32 * tri_el(j, j)];
                for (uint32_t k = 0; k < j; k++) {
                    const double lr = Ar[32 * tri_el(j, k)], li = Ai[32 * tri_el(j, k)];
                    d -= lr * lr + li * li;
                }
                if (!(d > 0.0) || !isfinite(d)) {
                    ok = false;
                    break;
                }
                const double ljj = sqrt(d), rl = 1.0 / ljj;
                Ar[32 * tri_el(j, j)] = ljj;
                Ai[32 * tri_el(j, j)] = 0.0;
                D[32 * j] = rl;
                for (uint32_t i = j + 1; i < n; i++) {
                    // (sg V_ij - sum_{k<j} L_ik conj(L_jk)) / L_jj
                    double sr = sg * Ar[32 * tri_el(i, j)], si = sg * Ai[32 * tri_el(i, j)];
                    for (uint32_t k = 0; k < j; k++) {
                        const double ar = Ar[32 * tri_el(i, k)], ai = Ai[32 * tri_el(i, k)];
                        const double br = Ar[32 * tri_el(j, k)], bi = Ai[32 * tri_el(j, k)];
                        sr -= ar * br + ai * bi;
                        si -= ai * br - ar * bi;
                    }
                    Ar[32 * tri_el(i, j)] = sr * rl;
                    Ai[32 * tri_el(i, j)] = si * rl;
                }
            }
        }
        if (ok) {
            // X_jj = 1 / L_jj, X_ij = -(sum_{j<=k<i} L_ik X_kj) / L_ii
            for (uint32_t j = 0; j < n; j++) {
                Ar[32 * tri_el(j, j)] = D[32 * j];
                for (uint32_t i = j + 1; i < n; i++) {
                    double ur = 0.0, ui = 0.0;
                    for (uint32_t k = j; k < i; k++) {
                        const double ar = Ar[32 * tri_el(i, k)], ai = Ai[32 * tri_el(i, k)];
                        const double xr = Ar[32 * tri_el(k, j)], xi = Ai[32 * tri_el(k, j)];
                        ur += ar * xr - ai * xi;
                        ui += ar * xi + ai * xr;
                    }
                    const double rli = D[32 * i];
                    Ar[32 * tri_el(i, j)] = -ur * rli;
                    Ai[32 * tri_el(i, j)] = -ui * rli;
                }
            }
            // W_ii = sum_{k >= i} |X_ki|^2 (D is free again)
            for (uint32_t i = 0; i < n; i++) {
                double w = 0.0;
                for (uint32_t k = i; k < n; k++) {
                    const double xr = Ar[32 * tri_el(k, i)], xi = Ai[32 * tri_el(k, i)];
                    w += xr * xr + xi * xi;
                }
                D[32 * i] = w;
            }
        }
        if (live) {
            for (uint32_t p = 0; p < NP; p++) {
                const uint32_t ij = __ldg(P.pairs + p), i = ij & 0xffffu, j = ij >> 16;
                double hre = 0.0, him = 0.0;   // (C^-1)_kk of the Re and Im components
                if (ok) {
                    const double wi = D[32 * i];
                    if (i == j) {
                        hre = N * (wi * wi);
                    } else {
                        double wr = 0.0, wm = 0.0;   // W_ij = sum_{k >= j} conj(X_ki) X_kj
                        for (uint32_t k = j; k < n; k++) {
                            const double ar = Ar[32 * tri_el(k, i)], ai = Ai[32 * tri_el(k, i)];
                            const double br = Ar[32 * tri_el(k, j)], bi = Ai[32 * tri_el(k, j)];
                            wr += ar * br + ai * bi;
                            wm += ar * bi - ai * br;
                        }
                        const double ww = wi * D[32 * j], re2 = wr * wr - wm * wm;
                        hre = 2.0 * N * (ww + re2);
                        him = 2.0 * N * (ww - re2);
                    }
                }
                for (int part = 0; part < 2; part++) {
                    if (part == 1 && i == j) break;
                    const uint32_t comp = part ? NP + p - i - 1 : p;
                    const double s2 = ok ? 1.0 / (part ? him : hre) : 0.0;
                    qtab[((size_t)fr * M + comp) * P.T + t] = ok ? (float)(12.0 * f * s2) : 0.0f;
                    if (s2_out) s2_out[smp * M + comp] = s2;
                }
            }
        }
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
    if (P.tslow) {
        // the post-acquisition reorder fused in: gather each output sample
        // from its time-slowest place (output writes stay coalesced)
        for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cplx;
             c += (uint64_t)gridDim.x * blockDim.x) {
            const uint32_t fp = (uint32_t)(c / P.T), t = (uint32_t)(c % P.T);
            const uint32_t f = fp / P.P, p = fp - f * P.P;
            out[c] = reduce_sample(__ldg(in + vis_src(P, c)), __ldg(P.pairs + p), f, t, P);
        }
        return;
    }
    for (uint64_t r = warp * RUN; r < n_cplx; r += nwarps * RUN) {
        uint32_t cnt = (uint32_t)(n_cplx - r < RUN ? n_cplx - r : RUN);
        if ((P.T & 1u) == 0) {
            // r is even and so is cnt (n_cplx = F P T is even): pairs of
            // samples (t, t + 1) of one product, four per lane loaded before
            // any is stored (out does not alias in), each placed in the cube
            // by division through precomputed multiply-high
            const uint4 *s4 = reinterpret_cast<const uint4 *>(in + r);
            uint4 *d4 = reinterpret_cast<uint4 *>(out + r);
            const uint32_t np = cnt / 2;
            for (uint32_t k0 = 0; k0 < np; k0 += 4 * 32) {
                uint4 v[4];
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    const uint32_t k = k0 + 32 * q + lane;
                    v[q] = k < np ? __ldg(s4 + k) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    const uint32_t k = k0 + 32 * q + lane;
                    if (k >= np) break;
                    const uint32_t c = (uint32_t)r + 2 * k;
                    const uint32_t fp = fastdiv(c, P.dT), t = c - fp * P.T;
                    const uint32_t f = fastdiv(fp, P.dP), p = fp - f * P.P;
                    d4[k] = reduce_pair(v[q], __ldg(P.pairs + p), f, t, P);
                }
            }
        } else {
            reduce_run(in + r, out + r, (uint32_t)r, cnt, P, lane);
        }
    }
}

// One warp per CTA, persistent.  Per block: wait for its bulk copy into `in`,
// round + transpose into `tmp`, start the next block's copy into `in`, then
// LZ4.  STAGED (the workspace holds two staging slots per warp): the block
// is encoded into a slot in global memory, its size published, and the
// PREVIOUS block placed, as the fast kernel does, so that the look-back
// rarely waits and no output buffer is needed; otherwise the block is
// encoded into `out`, placed by look-back and written out at once.
template <uint32_t MAXB, int LEVEL, bool STAGED>
__global__ void __launch_bounds__(32, MAXB <= 8192 ? 9 : 1)
    compress_kernel(const __grid_constant__ CodecArgs a)
{
    using L = CompPlan<MAXB, LEVEL>;
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *in = sm;
    uint8_t *tmp = sm + L::IN;
    uint8_t *out = tmp + L::TMP;  // not STAGED
    void *scratch = STAGED ? static_cast<void *>(tmp + L::TMP) : static_cast<void *>(out + L::OUT);
    uint64_t *bar = reinterpret_cast<uint64_t *>(static_cast<uint8_t *>(scratch) + r16(L::SCR));
    uint64_t *bar2 = bar + 1;  // STAGED: the placement copies
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(bar, 1);
        if (STAGED) mbar_init(bar2, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint8_t *slot0 = STAGED ? a.slots + (size_t)(2 * blockIdx.x) * L::SLOT : nullptr;
    uint8_t *slot1 = STAGED ? slot0 + L::SLOT : nullptr;
    uint32_t parity = 0, parity2 = 0;
    uint32_t ptile = ~0u, pcs = 0;  // STAGED: the block waiting to be placed, in slot1
    uint32_t tile = a.tile_begin + grab_tile(a.tile_counter, lane);
    bool pend = tile < a.tile_end && load_block_any(a, in, tile, bar, lane);
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
            pend = load_block_any(a, in, nxt, bar, lane);
        }
        if (STAGED) {
            const uint32_t cs =
                compress_encode<LEVEL, L::HBITS>(a, block_elems_of(a, tile), tmp, slot0, scratch, lane);
            lookback_publish(a.tile_state, tile, 4ull + cs, lane);
            if (ptile != ~0u) place_staged(a, ptile, slot1, pcs, tmp, bar2, parity2, lane);
            ptile = tile;
            pcs = cs;
            uint8_t *t = slot0;
            slot0 = slot1;
            slot1 = t;
        } else {
            compress_finish<MAXB, LEVEL>(a, tile, tmp, out, scratch, lane);
        }
        __syncwarp();
        tile = nxt;
    }
    if (STAGED && ptile != ~0u) place_staged(a, ptile, slot1, pcs, tmp, bar2, parity2, lane);
}


uint32_t compress_fast_smem_bytes(int level)
{
    return level >= 1 ? FastPlan<1>::BYTES : FastPlan<0>::BYTES;
}

uint32_t compress_fast_blocks_per_sm(int level, uint32_t es)
{
    int n = 0;
    const uint32_t smem = compress_fast_smem_bytes(level);
    cudaError_t e;
    if (es == 8)
        e = level >= 1
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<1, 8>, 32, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<0, 8>, 32, smem);
    else if (es == 2)
        e = level >= 1
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<1, 2>, 32, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<0, 2>, 32, smem);
    else
        e = level >= 1
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<1, 4>, 32, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, compress_fast_kernel<0, 4>, 32, smem);
    return e == cudaSuccess && n > 0 ? (uint32_t)n : 1u;
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
            const uint32_t x = src[2 * vis_src(a.vis, lane >> 1) + (lane & 1)];
            const uint32_t u = reduce_component_at(x, lane, a.vis);
            for (int k = 0; k < 4; k++) a.out[12 + 4 * lane + k] = (uint8_t)(u >> (8 * k));
        }
    } else {
        for (uint32_t k = lane; k < tb; k += 32) a.out[12 + k] = a.in[k];
    }
    if (lane == 0) *a.out_bytes = 12 + tb;
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
            if (ES == 2)
                unshuffle2_inplace(dec, Bb, lane);
            else if (ES == 4)
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

// Decompress with ONE shared buffer per warp, for blocks of at most 8 KiB whose
// un-transpose fits in registers (2-, 4- and 8-byte elements): LZ4 in-place
// decoding, the block's compressed bytes loaded at the end of the buffer and
// the output written from its start.  For any valid LZ4 block the output
// written so far never catches up with the unread input: ahead of any
// literal run, the rest of the stream holds at most 2 + 2 S / 255 bytes more
// than it produces (a token, length bytes and a final literal run; every
// match adds at least one more byte than its three), about 72 bytes for
// S = 8192, and the image starts at least 113 bytes later than that needs.
// Half the shared memory of decompress_kernel: 16 resident warps per SM
// instead of 13, at the cost of the next block's copy starting only once
// this block's store has read the buffer.

template <int ES>
__global__ void __launch_bounds__(32, 20) decompress_inplace_kernel(const __grid_constant__ CodecArgs a)
{
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *buf = sm;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + INPLACE_BUF);
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;
    bool header_checked = false;
    uint32_t tile = grab_tile(a.tile_counter, lane);
    DecLoad ld{};
    if (tile < a.nb) ld = dec_issue(a, tile, buf, bar, lane, INPLACE_BUF);
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
        uint8_t *comp = buf + cur.off;
        bool good = cur.ok;
        if (good) {
            if (cur.eidx != ~0u) comp[cur.eidx] = cur.ebyte;
            __syncwarp();
            good = get_be32(comp + cur.delta) == cur.clen &&
                   lz4_decode_warp(comp, cur.delta + 4, cur.clen, buf, S) == 0;
        }
        if (!good && lane == 0) set_status(a.status, BSGPU_ERR_CORRUPT);
        __syncwarp();
        uint8_t *dst = a.out + (uint64_t)tile * a.B * a.es;
        if (good && unshuffle_inplace_ok(ES, Bb)) {
            if (ES == 2)
                unshuffle2_inplace(buf, Bb, lane);
            else if (ES == 4)
                unshuffle4_inplace(buf, Bb, lane);
            else
                unshuffle8_inplace(buf, Bb, lane);
            __syncwarp();
            if ((S & 15u) == 0 && ((uintptr_t)dst & 15u) == 0) {
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    bulk_s2g(dst, buf, S);
                    bulk_commit();
                }
            } else {
                for (uint32_t k = lane; k < S; k += 32) dst[k] = buf[k];
            }
        } else if (good) {
            unshuffle_generic(buf, dst, Bb, a.es, lane);  // a shortened last block
        }
        if (tile + 1 == a.nb) {
            const uint32_t tb = a.tail_elems * a.es;
            const uint64_t first = (a.n_elem - a.tail_elems) * a.es;
            if (a.in_bytes >= tb)
                for (uint32_t k = lane; k < tb; k += 32)
                    a.out[first + k] = a.in[a.in_bytes - tb + k];
        }
        __syncwarp();
        // the next block's bytes go into the same buffer once the store has read it
        if (lane == 0) bulk_wait_read0();
        __syncwarp();
        ld = DecLoad{};
        if (nxt < a.nb) {
            fence_proxy_async_smem();
            __syncwarp();
            ld = dec_issue(a, nxt, buf, bar, lane, INPLACE_BUF);
        }
        tile = nxt;
    }
    if (lane == 0) bulk_wait0();
    __syncwarp();
}

// In-place decoding for the shapes the 8 KiB kernel does not take (blocks
// over 8 KiB, 1-byte elements): one buffer per warp with the block's
// compressed image near its end and the bit-rows decoded from its start,
// un-transposed from there straight into the output, which is 16-byte
// aligned for every block (the caller checks B * es).  The margin argument
// above holds for any S: the LZ4 bytes must start at least 2 + 2 S / 255
// bytes after S - clen, and dec_issue puts them at least E - clen - 47
// bytes in (E the buffer size), so E >= S + 2 S / 255 + 49 suffices
// (inplace_any_buf gives S + 2 S / 255 + 160).  Half the shared memory of
// decompress_kernel, which holds the compressed and the decoded block apart:
// twice the resident warps or more.
template <uint32_t MAXB>
__global__ void __launch_bounds__(32, MAXB <= 8192 ? 20 : (MAXB <= 16384 ? 12 : (MAXB <= 32768 ? 6 : 3)))
    decompress_inplace_any_kernel(const __grid_constant__ CodecArgs a)
{
    constexpr uint32_t BUF = inplace_any_buf(MAXB);
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *buf = sm;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + BUF);
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;
    bool header_checked = false;
    uint32_t tile = grab_tile(a.tile_counter, lane);
    DecLoad ld{};
    if (tile < a.nb) ld = dec_issue(a, tile, buf, bar, lane, BUF);
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
        uint8_t *comp = buf + cur.off;
        bool good = cur.ok;
        if (good) {
            if (cur.eidx != ~0u) comp[cur.eidx] = cur.ebyte;
            __syncwarp();
            good = get_be32(comp + cur.delta) == cur.clen &&
                   lz4_decode_warp(comp, cur.delta + 4, cur.clen, buf, S) == 0;
        }
        if (!good && lane == 0) set_status(a.status, BSGPU_ERR_CORRUPT);
        __syncwarp();
        if (good) unshuffle_block(buf, a.out + (uint64_t)tile * a.B * a.es, Bb, a.es, lane);
        if (tile + 1 == a.nb) {
            const uint32_t tb = a.tail_elems * a.es;
            const uint64_t first = (a.n_elem - a.tail_elems) * a.es;
            if (a.in_bytes >= tb)
                for (uint32_t k = lane; k < tb; k += 32)
                    a.out[first + k] = a.in[a.in_bytes - tb + k];
        }
        // the next block's bytes go into the buffer once the un-transpose has read it
        fence_proxy_async_smem();
        __syncwarp();
        ld = DecLoad{};
        if (nxt < a.nb) ld = dec_issue(a, nxt, buf, bar, lane, BUF);
        tile = nxt;
    }
}

uint32_t decompress_inplace_any_smem_bytes(uint32_t maxb)
{
    return inplace_any_buf(maxb) + 16;
}

uint32_t decompress_inplace_blocks_per_sm(uint32_t es)
{
    int n = 0;
    const uint32_t smem = INPLACE_BUF + 16;
    cudaError_t e = es == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decompress_inplace_kernel<2>, 32, smem)
                  : es == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decompress_inplace_kernel<4>, 32, smem)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, decompress_inplace_kernel<8>, 32, smem);
    return e == cudaSuccess && n > 0 ? (uint32_t)n : 1u;
}

static_assert(SEG_WS_BYTES >= SEG_WS_REC, "workspace of the parallel index recovery");

// Parallel recovery of the block index, phase 1: warp k takes the first
// plausible block start of segment k and walks the chain across the
// segment and SEG_M positions past it.
__global__ void __launch_bounds__(128) chain_seg_find_kernel(const __grid_constant__ CodecArgs a,
                                                            SegRec *recs, uint32_t K, uint64_t Z,
                                                            uint32_t maxlen)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= K) return;
    const uint64_t tail_b = (uint64_t)a.tail_elems * a.es;
    SegRec *rec = recs + k;
    uint32_t c = 0, nh = 0, na = 0;
    bool ok = false;
    if (a.in_bytes >= 12 + tail_b) {
        const uint64_t end = a.in_bytes - tail_b;
        const uint64_t lo = 12 + (uint64_t)k * Z;
        const uint64_t hi = (k + 1 == K || lo + Z > end) ? end : lo + Z;
        uint64_t f = k == 0 ? 12ull : ~0ull;
        // candidates in address order, 128 per step: lane l tests the four
        // offsets c0 + 4 l .. c0 + 4 l + 3 from seven bytes
        for (uint64_t c0 = lo; k && c0 < hi && f == ~0ull; c0 += 128) {
            const uint64_t p = c0 + 4 * lane;
            uint32_t b[7];
#pragma unroll
            for (int t = 0; t < 7; t++) b[t] = p + t < end ? __ldg(a.in + p + t) : 0u;
            uint32_t mine = 0;
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const uint64_t q = p + t;
                const uint32_t len = (b[t] << 24) | (b[t + 1] << 16) | (b[t + 2] << 8) | b[t + 3];
                if (q < hi && q + 4 <= end && len >= 1 && len <= maxlen && q + 4 + len <= end)
                    mine |= 1u << t;
            }
            uint32_t m = __ballot_sync(FULL, mine != 0);
            while (m) {   // deeper checks in address order (the warp in step)
                const uint32_t l = __ffs(m) - 1;
                m &= m - 1;
                uint32_t bits = __shfl_sync(FULL, mine, l);
                while (bits) {
                    const uint32_t t = __ffs(bits) - 1;
                    bits &= bits - 1;
                    const uint64_t q = c0 + 4 * l + t;
                    if (seg_plausible(a.in, q, end, maxlen, SEG_DEPTH)) {
                        f = q;
                        break;
                    }
                }
                if (f != ~0ull) break;
            }
        }
        ok = f != ~0ull;
        uint64_t D = f;
        // each step advances D by 5 bytes at least; past the segment at most
        // SEG_M more steps
        while (ok && D < end) {
            if (D < hi) {
                if (nh < SEG_M && lane == 0) rec->head[nh] = D;
                if (nh < SEG_M) nh++;
                c++;
            } else {
                if (na == SEG_M) break;
                if (lane == 0) rec->after[na] = D;
                na++;
            }
            if (D + 4 > end) {
                ok = false;
                break;
            }
            const uint32_t len = stream_be32(a.in, D);
            if (len < 1 || len > maxlen || D + 4 + len > end) {
                ok = false;
                break;
            }
            D += 4ull + len;
        }
        if (ok && D == end && na < SEG_M) {   // the chain reached the area's end
            if (lane == 0) rec->after[na] = D;
            na++;
        }
    }
    if (lane == 0) {
        rec->c = c;
        rec->nh = nh;
        rec->na = na;
        rec->ok = ok ? 1u : 0u;
    }
}

// Phase 2 (one CTA of 1024 threads): warp k - 1's positions past its
// segment must meet warp k's first positions within SEG_M steps; the
// meeting point corrects warp k's count (the true blocks before it that
// start in segment k, minus warp k's own blocks before it); the counts must
// add up to nb and the last walk must end at the area's end.  Then the
// counts' exclusive scan numbers each segment's first block.
__global__ void __launch_bounds__(1024) chain_seg_scan_kernel(const __grid_constant__ CodecArgs a,
                                                             SegRec *recs, uint32_t K, uint64_t Z,
                                                             uint32_t *verified)
{
    __shared__ uint64_t part[1024];
    const uint32_t t = threadIdx.x;
    const uint64_t tail_b = (uint64_t)a.tail_elems * a.es;
    const uint64_t end = a.in_bytes >= 12 + tail_b ? a.in_bytes - tail_b : 0;
    bool good = end != 0;
    uint64_t cnt = 0;
    uint64_t cnt_k[2] = {0, 0}, start_k[2] = {0, 0};
    for (uint32_t k = 2 * t, u = 0; u < 2 && k < K; k++, u++) {
        const SegRec &r = recs[k];
        good = good && r.ok;
        const uint64_t hi = (k + 1 == K || 12 + (uint64_t)(k + 1) * Z > end) ? end
                                                                            : 12 + (uint64_t)(k + 1) * Z;
        uint64_t ck = r.c, st = 12;
        if (k > 0) {
            const SegRec &q = recs[k - 1];
            // first position past segment k - 1 that warp k's walk also visits
            uint32_t hit_i = SEG_M, hit_j = 0;
            for (uint32_t i = 0; i < q.na && hit_i == SEG_M; i++)
                for (uint32_t j = 0; j < r.nh; j++)
                    if (q.after[i] == r.head[j]) {
                        hit_i = i;
                        hit_j = j;
                        break;
                    }
            // the true blocks before the meeting point must start in this segment
            good = good && hit_i < SEG_M && (hit_i == 0 || q.after[hit_i - 1] < hi);
            if (hit_i < SEG_M) {
                ck = hit_i + (uint64_t)r.c - hit_j;
                st = q.na ? q.after[0] : 0;
            }
        } else {
            good = good && r.nh > 0 && r.head[0] == 12;
        }
        if (k + 1 == K) good = good && r.na > 0 && r.after[0] == end;
        cnt_k[u] = ck;
        start_k[u] = st;
        cnt += ck;
    }
    part[t] = cnt;
    __syncthreads();
    for (uint32_t d = 1; d < 1024; d <<= 1) {   // inclusive scan (Hillis-Steele)
        const uint64_t v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint64_t base = part[t] - cnt;
    for (uint32_t k = 2 * t, u = 0; u < 2 && k < K; k++, u++) {
        recs[k].base = base;
        recs[k].start = start_k[u];
        recs[k].c = (uint32_t)cnt_k[u];
        base += cnt_k[u];
    }
    const int all = __syncthreads_and(good ? 1 : 0);
    if (t == 0) *verified = (all && part[1023] == a.nb) ? 1u : 0u;
}

// Phase 3: each segment writes the offsets of the true blocks starting in
// it, walking the chain from its true first block.
__global__ void __launch_bounds__(128) chain_seg_write_kernel(const __grid_constant__ CodecArgs a,
                                                             const SegRec *recs, uint32_t K,
                                                             const uint32_t *verified,
                                                             uint64_t *offsets)
{
    const uint32_t k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= K || !*verified || (threadIdx.x & 31u) != 0) return;
    const SegRec &r = recs[k];
    uint64_t D = r.start;
    for (uint32_t i = 0; i < r.c; i++) {
        offsets[r.base + i] = D;
        D += 4ull + stream_be32(a.in, D);
    }
}

// Block offsets by walking the chain of 4-byte length fields: one warp, the
// stream staged through shared memory (chain_walk_staged); skipped when the
// parallel recovery has verified its index (*done set).
__global__ void __launch_bounds__(32, 1) chain_walk_kernel(const __grid_constant__ CodecArgs a,
                                                           uint64_t *offsets, const uint32_t *done)
{
    extern __shared__ __align__(128) uint8_t sm[];
    if (done && *done) return;
    const uint32_t lane = threadIdx.x & 31u;
    bool timely = true;
    const bool ok = chain_walk_staged(a.in, a.in_bytes, a.nb, (uint64_t)a.tail_elems * a.es,
                                      offsets, sm, lane, timely);
    if (lane == 0 && !timely) set_status(a.status, BSGPU_ERR_TIMEOUT);
    else if (lane == 0 && !ok) set_status(a.status, BSGPU_ERR_CORRUPT);
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
// Standalone Bitshuffle of blocks larger than 16 KiB (4- or 8-byte elements,
// a multiple of 1024 elements): a block's groups of 32 elements are
// independent, so the unit of work is a tile of 32 groups (1024 elements;
// lane l takes group l), whatever the block size; only the stride of a
// bit-row (B / 32 words) depends on it.  Forward: the tile is bulk-copied
// into shared memory (the next one prefetched), each lane transposes its
// group in registers and row r of the tile goes out as one coalesced
// 128-byte store per row.  Inverse: lane l loads word l of each of the
// tile's rows (coalesced), transposes and writes its group to shared
// memory, and the tile is bulk-stored.  A warp holds two tiles (8 or 16
// KiB) instead of whole blocks, so many warps fit on an SM.  Full blocks
// only; the shortened last block and the verbatim tail take shuffle_kernel.
constexpr uint32_t TILE_ELEMS = 1024;

template <int ES, bool INV>
__global__ void __launch_bounds__(32, 16) shuffle_tile_kernel(const __grid_constant__ CodecArgs a,
                                                              uint32_t nfull)
{
    constexpr uint32_t TB = TILE_ELEMS * ES;   // bytes of a tile
    extern __shared__ __align__(128) uint8_t sm[];
    uint8_t *buf[2] = {sm, sm + TB};
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + 2 * TB);
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const uint32_t tpb = a.B / TILE_ELEMS;             // tiles per block
    const uint64_t items = (uint64_t)nfull * tpb;
    const uint32_t rs = a.B / 32;                       // words per bit-row
    const uint32_t rot = lane & (ES == 4 ? 7u : 15u);
    uint32_t parity[2] = {0u, 0u};
    auto tile_src = [&](uint64_t it) {   // the tile's bytes in the element order
        const uint64_t b = it / tpb, t = it - b * tpb;
        return (b * a.B + t * TILE_ELEMS) * ES;
    };
    uint64_t it = blockIdx.x;
    int cur = 0;
    if (!INV && it < items && lane == 0) {
        mbar_arrive_expect_tx(&bar[0], TB);
        bulk_g2s(buf[0], a.in + tile_src(it), TB, &bar[0]);
    }
    for (; it < items; it += gridDim.x) {
        const uint64_t nxt = it + gridDim.x;
        const uint64_t b = it / tpb, t = it - b * tpb;
        if (!INV) {
            if (!mbar_wait_bounded(&bar[cur], parity[cur]) && lane == 0)
                set_status(a.status, BSGPU_ERR_TIMEOUT);
            parity[cur] ^= 1u;
            if (nxt < items && lane == 0) {
                // the other buffer's generic reads finished before this step
                mbar_arrive_expect_tx(&bar[cur ^ 1], TB);
                bulk_g2s(buf[cur ^ 1], a.in + tile_src(nxt), TB, &bar[cur ^ 1]);
            }
            // rows of the tile: words [t * 32, t * 32 + 32) of each bit-row
            uint32_t *o32 = reinterpret_cast<uint32_t *>(a.out + b * a.B * ES) + t * 32 + lane;
            const uint8_t *grp = buf[cur] + (size_t)(ES * 32) * lane;
            if (ES == 4) {
                uint32_t v[32];
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const uint4 q = *reinterpret_cast<const uint4 *>(grp + 16u * ((k + rot) & 7u));
                    v[4 * k] = q.x;
                    v[4 * k + 1] = q.y;
                    v[4 * k + 2] = q.z;
                    v[4 * k + 3] = q.w;
                }
                transpose32(v);
#pragma unroll
                for (int r = 0; r < 32; r++) o32[(size_t)r * rs] = rotl(v[r], 4u * rot);
            } else {
                uint32_t lo[32], hi[32];
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    const uint4 q = *reinterpret_cast<const uint4 *>(grp + 16u * ((k + rot) & 15u));
                    lo[2 * k] = q.x;
                    hi[2 * k] = q.y;
                    lo[2 * k + 1] = q.z;
                    hi[2 * k + 1] = q.w;
                }
                transpose32(lo);
#pragma unroll
                for (int r = 0; r < 32; r++) o32[(size_t)r * rs] = rotl(lo[r], 2u * rot);
                transpose32(hi);
#pragma unroll
                for (int r = 0; r < 32; r++) o32[(size_t)(32 + r) * rs] = rotl(hi[r], 2u * rot);
            }
            __syncwarp();
            fence_proxy_async_smem();   // the reads of buf[cur] before its next bulk write
            __syncwarp();
        } else {
            const uint32_t *i32 =
                reinterpret_cast<const uint32_t *>(a.in + b * a.B * ES) + t * 32 + lane;
            // the previous bulk store from this buffer must have read it
            if (lane == 0) bulk_wait_read0();
            __syncwarp();
            uint8_t *grp = buf[cur] + (size_t)(ES * 32) * lane;
            if (ES == 4) {
                uint32_t v[32];
#pragma unroll
                for (int r = 0; r < 32; r++) v[r] = rotr(__ldg(i32 + (size_t)r * rs), 4u * rot);
                transpose32(v);
#pragma unroll
                for (int k = 0; k < 8; k++)
                    *reinterpret_cast<uint4 *>(grp + 16u * ((k + rot) & 7u)) =
                        make_uint4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            } else {
                uint32_t lo[32], hi[32];
#pragma unroll
                for (int r = 0; r < 32; r++) {
                    lo[r] = rotr(__ldg(i32 + (size_t)r * rs), 2u * rot);
                    hi[r] = rotr(__ldg(i32 + (size_t)(32 + r) * rs), 2u * rot);
                }
                transpose32(lo);
                transpose32(hi);
#pragma unroll
                for (int k = 0; k < 16; k++)
                    *reinterpret_cast<uint4 *>(grp + 16u * ((k + rot) & 15u)) =
                        make_uint4(lo[2 * k], hi[2 * k], lo[2 * k + 1], hi[2 * k + 1]);
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                bulk_s2g(a.out + tile_src(it), buf[cur], TB);
                bulk_commit();
            }
        }
        cur ^= 1;
    }
    if (INV && lane == 0) bulk_wait0();
    // the verbatim tail, when every block is full
    if (nfull == a.nb && blockIdx.x == 0) {
        const uint64_t first = (a.n_elem - a.tail_elems) * ES;
        for (uint32_t k = lane; k < a.tail_elems * ES; k += 32) a.out[first + k] = a.in[first + k];
    }
}

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
    uint32_t tile = a.tile_begin + blockIdx.x;   // tile_begin: blocks before it are done
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
cudaError_t launch_vis_compensation(const void *vis, const VisParams &P, uint32_t n_freq,
                                    double f, double N, cudaStream_t s)
{
    const uint64_t work = (uint64_t)n_freq * ((P.T + 1023) / 1024);
    const uint32_t grid = (uint32_t)(work < 8192 ? work : 8192);
    vis_compensation_kernel<<<grid ? grid : 1, 256, 0, s>>>(vis, P, const_cast<float *>(P.cft),
                                                            n_freq, f, N);
    return cudaGetLastError();
}

uint32_t full_noise_smem_bytes(uint32_t n_in)
{
    return (2u * (n_in * (n_in + 1) / 2) + n_in) * 32u * 8u;
}

cudaError_t launch_full_noise(const void *vis, const VisParams &P, uint32_t n_freq, double f,
                              double N, double *s2, cudaStream_t s)
{
    const uint32_t smem = full_noise_smem_bytes(P.n_in);
    cudaError_t e = cudaFuncSetAttribute(full_noise_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148, per = 1;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, full_noise_kernel, 32, smem);
    const uint64_t ctas = ((uint64_t)n_freq * P.T + 31) / 32;
    const uint64_t want = (uint64_t)sms * (per > 0 ? per : 1);
    const uint32_t grid = (uint32_t)(ctas < want ? ctas : want);
    full_noise_kernel<<<grid ? grid : 1, 32, smem, s>>>(vis, P, n_freq, f, N, s2);
    return cudaGetLastError();
}

cudaError_t launch_vis_tables(const float *vis, const VisParams &V, uint32_t n_freq,
                              cudaStream_t s)
{
    uint64_t n = (uint64_t)n_freq * V.n_in * V.T;
    uint64_t P = (uint64_t)V.n_in * (V.n_in + 1) / 2;
    uint64_t work = n > P ? n : P;
    uint32_t blocks = (uint32_t)((work + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks == 0) blocks = 1;
    vis_tables_kernel<<<blocks, 256, 0, s>>>(vis, V, n_freq);
    return cudaGetLastError();
}

// Post-acquisition reorder (Sec. 2): [T][S] elements (time slowest, the
// order an instrument writes) to [S][T] (time fastest), through 32 x 32
// tiles in shared memory so that reads and writes are both coalesced.
template <typename E>
__global__ void __launch_bounds__(256) reorder_time_kernel(const E *__restrict__ in,
                                                           E *__restrict__ out, uint64_t T,
                                                           uint64_t S)
{
    __shared__ E tile[32][33];
    const uint64_t ntx = (S + 31) / 32, nty = (T + 31) / 32;
    for (uint64_t b = blockIdx.x; b < ntx * nty; b += gridDim.x) {
        const uint64_t s0 = (b % ntx) * 32, t0 = (b / ntx) * 32;
        __syncthreads();
        for (uint32_t k = threadIdx.y; k < 32; k += blockDim.y) {
            const uint64_t t = t0 + k, sx = s0 + threadIdx.x;
            if (t < T && sx < S) tile[k][threadIdx.x] = in[t * S + sx];
        }
        __syncthreads();
        for (uint32_t k = threadIdx.y; k < 32; k += blockDim.y) {
            const uint64_t sx = s0 + k, t = t0 + threadIdx.x;
            if (t < T && sx < S) out[sx * T + t] = tile[threadIdx.x][k];
        }
    }
}

// The same for a short time axis (T <= 32): a tile is all T time rows of 64
// series, read row by row (64 consecutive elements each) and written as the
// tile's one contiguous stretch of output (64 series of T samples), element
// o of the stretch from tile[o mod T][o / T]; the row pitch of 65 elements
// keeps those transposed reads free of bank conflicts.
template <typename E>
__global__ void __launch_bounds__(256) reorder_time_short_kernel(const E *__restrict__ in,
                                                                 E *__restrict__ out, uint32_t T,
                                                                 uint64_t S)
{
    constexpr uint32_t W = 64;
    __shared__ E tile[32][W + 1];
    const uint32_t tid = threadIdx.x, nt = blockDim.x;
    const uint64_t ntiles = (S + W - 1) / W;
    for (uint64_t b = blockIdx.x; b < ntiles; b += gridDim.x) {
        const uint64_t s0 = b * W;
        const uint32_t w = S - s0 < W ? (uint32_t)(S - s0) : W;   // series in this tile
        __syncthreads();
        for (uint32_t e = tid; e < T * W; e += nt) {
            const uint32_t t = e / W, x = e % W;
            if (x < w) tile[t][x] = in[(uint64_t)t * S + s0 + x];
        }
        __syncthreads();
        E *o = out + s0 * T;
        // element e = x T + t of the stretch; (t, x) advance by nt per step
        const uint32_t qn = nt / T, rn = nt % T;
        uint32_t t = tid % T, x = tid / T;
        for (uint32_t e = tid; e < w * T; e += nt) {
            o[e] = tile[t][x];
            t += rn;
            x += qn;
            if (t >= T) {
                t -= T;
                x++;
            }
        }
    }
}

cudaError_t launch_reorder_time(const void *in, void *out, uint64_t T, uint64_t S, uint32_t es,
                                cudaStream_t s)
{
    if (T >= 1 && T <= 32) {
        const uint64_t tiles = (S + 63) / 64;
        const uint32_t grid = (uint32_t)(tiles < 65536 ? (tiles ? tiles : 1) : 65536);
        const uint32_t t32 = (uint32_t)T;
        switch (es) {
        case 1: reorder_time_short_kernel<<<grid, 256, 0, s>>>((const uint8_t *)in, (uint8_t *)out, t32, S); break;
        case 2: reorder_time_short_kernel<<<grid, 256, 0, s>>>((const uint16_t *)in, (uint16_t *)out, t32, S); break;
        case 4: reorder_time_short_kernel<<<grid, 256, 0, s>>>((const uint32_t *)in, (uint32_t *)out, t32, S); break;
        default: reorder_time_short_kernel<<<grid, 256, 0, s>>>((const uint2 *)in, (uint2 *)out, t32, S); break;
        }
        return cudaGetLastError();
    }
    const uint64_t tiles = ((S + 31) / 32) * ((T + 31) / 32);
    const uint32_t grid = (uint32_t)(tiles < 65536 ? (tiles ? tiles : 1) : 65536);
    const dim3 blk(32, 8);
    switch (es) {
    case 1: reorder_time_kernel<<<grid, blk, 0, s>>>((const uint8_t *)in, (uint8_t *)out, T, S); break;
    case 2: reorder_time_kernel<<<grid, blk, 0, s>>>((const uint16_t *)in, (uint16_t *)out, T, S); break;
    case 4: reorder_time_kernel<<<grid, blk, 0, s>>>((const uint32_t *)in, (uint32_t *)out, T, S); break;
    default: reorder_time_kernel<<<grid, blk, 0, s>>>((const uint2 *)in, (uint2 *)out, T, S); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_precision(const float *in, float *out, uint64_t n_cplx,
                                    const VisParams &v, uint32_t grid, cudaStream_t s)
{
    reduce_precision_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const uint2 *>(in),
                                                 reinterpret_cast<uint2 *>(out), n_cplx, v);
    return cudaGetLastError();
}

template <typename K>
cudaError_t launch_tiles(K kernel, uint32_t smem, uint32_t grid, cudaStream_t s, const CodecArgs &a,
                         uint32_t nfull)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, 32, smem, s>>>(a, nfull);
    return cudaGetLastError();
}

cudaError_t launch_shuffle(const CodecArgs &a_in, bool inverse, uint32_t maxb, uint32_t grid,
                           cudaStream_t s)
{
    CodecArgs a = a_in;
    if (maxb > 16384 && (a.es == 4 || a.es == 8) && a.B % TILE_ELEMS == 0 && a.nb) {
        // full blocks by tiles; the shortened last block (if any) and the
        // tail below
        const uint32_t nfull = a.last_B == a.B ? a.nb : a.nb - 1;
        if (nfull) {
            const uint32_t tsm = 2 * TILE_ELEMS * a.es + 16;
            int dev = 0, sms = 148;
            if (cudaGetDevice(&dev) == cudaSuccess)
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const uint64_t items = (uint64_t)nfull * (a.B / TILE_ELEMS);
            uint64_t g = (uint64_t)sms * 16;
            if (g > items) g = items;
            cudaError_t e;
            if (a.es == 4)
                e = inverse ? launch_tiles(shuffle_tile_kernel<4, true>, tsm, (uint32_t)g, s, a, nfull)
                            : launch_tiles(shuffle_tile_kernel<4, false>, tsm, (uint32_t)g, s, a, nfull);
            else
                e = inverse ? launch_tiles(shuffle_tile_kernel<8, true>, tsm, (uint32_t)g, s, a, nfull)
                            : launch_tiles(shuffle_tile_kernel<8, false>, tsm, (uint32_t)g, s, a, nfull);
            if (e != cudaSuccess || nfull == a.nb) return e;
        }
        a.tile_begin = nfull;   // the shortened last block and the tail
        grid = 1;
    }
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

template <bool STAGED>
cudaError_t launch_compress_t(const CodecArgs &a, uint32_t maxb, uint32_t grid, cudaStream_t s)
{
    const uint32_t smem = compress_smem_bytes(maxb, a.level, STAGED);
    if (a.level >= 1) {
        if (maxb <= 8192) return launch_warp_kernel(compress_kernel<8192, 1, STAGED>, smem, grid, s, a);
        if (maxb <= 16384) return launch_warp_kernel(compress_kernel<16384, 1, STAGED>, smem, grid, s, a);
        if (maxb <= 32768) return launch_warp_kernel(compress_kernel<32768, 1, STAGED>, smem, grid, s, a);
        return launch_warp_kernel(compress_kernel<65536, 1, STAGED>, smem, grid, s, a);
    }
    if (maxb <= 8192) return launch_warp_kernel(compress_kernel<8192, 0, STAGED>, smem, grid, s, a);
    if (maxb <= 16384) return launch_warp_kernel(compress_kernel<16384, 0, STAGED>, smem, grid, s, a);
    if (maxb <= 32768) return launch_warp_kernel(compress_kernel<32768, 0, STAGED>, smem, grid, s, a);
    return launch_warp_kernel(compress_kernel<65536, 0, STAGED>, smem, grid, s, a);
}

cudaError_t launch_compress(const CodecArgs &a, uint32_t maxb, uint32_t grid, cudaStream_t s)
{
    return a.slots ? launch_compress_t<true>(a, maxb, grid, s) : launch_compress_t<false>(a, maxb, grid, s);
}

cudaError_t launch_compress_fast(const CodecArgs &a, uint32_t grid, cudaStream_t s)
{
    const uint32_t smem = compress_fast_smem_bytes(a.level);
    if (a.es == 8)
        return a.level >= 1 ? launch_warp_kernel(compress_fast_kernel<1, 8>, smem, grid, s, a)
                            : launch_warp_kernel(compress_fast_kernel<0, 8>, smem, grid, s, a);
    if (a.es == 2)
        return a.level >= 1 ? launch_warp_kernel(compress_fast_kernel<1, 2>, smem, grid, s, a)
                            : launch_warp_kernel(compress_fast_kernel<0, 2>, smem, grid, s, a);
    if (a.vis.enabled && (a.vis.is_int || a.vis.cft || a.vis.qtab))
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
    if (maxb <= 8192 && (a.es == 2 || a.es == 4 || a.es == 8)) {
        const uint32_t sm1 = INPLACE_BUF + 16;
        if (a.es == 2) return launch_warp_kernel(decompress_inplace_kernel<2>, sm1, grid, s, a);
        if (a.es == 4) return launch_warp_kernel(decompress_inplace_kernel<4>, sm1, grid, s, a);
        return launch_warp_kernel(decompress_inplace_kernel<8>, sm1, grid, s, a);
    }
    if (maxb <= 8192) {
        if (a.es == 2) return launch_warp_kernel(decompress_kernel<8192, 2>, smem, grid, s, a);
        if (a.es == 4) return launch_warp_kernel(decompress_kernel<8192, 4>, smem, grid, s, a);
        if (a.es == 8) return launch_warp_kernel(decompress_kernel<8192, 8>, smem, grid, s, a);
        return launch_warp_kernel(decompress_kernel<8192, 0>, smem, grid, s, a);
    }
    if (maxb <= 16384) return launch_warp_kernel(decompress_kernel<16384, 0>, smem, grid, s, a);
    if (maxb <= 32768) return launch_warp_kernel(decompress_kernel<32768, 0>, smem, grid, s, a);
    return launch_warp_kernel(decompress_kernel<65536, 0>, smem, grid, s, a);
}

cudaError_t launch_decompress_inplace_any(const CodecArgs &a, uint32_t maxb, uint32_t grid,
                                          cudaStream_t s)
{
    const uint32_t smem = decompress_inplace_any_smem_bytes(maxb);
    if (maxb <= 8192) return launch_warp_kernel(decompress_inplace_any_kernel<8192>, smem, grid, s, a);
    if (maxb <= 16384) return launch_warp_kernel(decompress_inplace_any_kernel<16384>, smem, grid, s, a);
    if (maxb <= 32768) return launch_warp_kernel(decompress_inplace_any_kernel<32768>, smem, grid, s, a);
    return launch_warp_kernel(decompress_inplace_any_kernel<65536>, smem, grid, s, a);
}

cudaError_t launch_chain_walk(const CodecArgs &a, uint64_t *offsets, void *seg_ws,
                              cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(chain_walk_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WALK_SMEM);
    if (e != cudaSuccess) return e;
    uint32_t *verified = nullptr;
    if (seg_ws) {
        // the parallel recovery: segments of at least four largest blocks
        const uint32_t S = (uint32_t)((uint64_t)a.B * a.es);
        const uint32_t maxlen = S + S / 255u + 16u;
        const uint64_t tail_b = (uint64_t)a.tail_elems * a.es;
        const uint64_t area = a.in_bytes > 12 + tail_b ? a.in_bytes - 12 - tail_b : 0;
        uint64_t K = area / ((SEG_M + 1ull) * (maxlen + 4));
        if (K > SEG_MAX) K = SEG_MAX;
        if (K < 1) K = 1;
        const uint64_t Z = (area + K - 1) / K;
        verified = reinterpret_cast<uint32_t *>(seg_ws);
        SegRec *recs = reinterpret_cast<SegRec *>((uint8_t *)seg_ws + 256);
        const uint32_t ctas = (uint32_t)((K + 3) / 4);
        chain_seg_find_kernel<<<ctas, 128, 0, s>>>(a, recs, (uint32_t)K, Z, maxlen);
        chain_seg_scan_kernel<<<1, 1024, 0, s>>>(a, recs, (uint32_t)K, Z, verified);
        chain_seg_write_kernel<<<ctas, 128, 0, s>>>(a, recs, (uint32_t)K, verified, offsets);
    }
    chain_walk_kernel<<<1, 32, WALK_SMEM, s>>>(a, offsets, verified);
    return cudaGetLastError();
}

}  // namespace bsg
