// Device helpers shared by the bsgpu kernels (sm_103a).
//
// Bit manipulation helpers are __host__ __device__ so that the host-side
// unit test (tests/host_emu/device_code_test.cu) can check them on a CPU.
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/bsgpu.h"

#define BSG_HD __host__ __device__ __forceinline__
#define BSG_D __device__ __forceinline__

namespace bsg {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// byte permute and funnel shifts (device intrinsics, portable host versions)
// ---------------------------------------------------------------------------
BSG_HD uint32_t bperm(uint32_t a, uint32_t b, uint32_t sel)
{
#ifdef __CUDA_ARCH__
    return __byte_perm(a, b, sel);
#else
    uint64_t x = (uint64_t)a | ((uint64_t)b << 32);
    uint32_t r = 0;
    for (int k = 0; k < 4; k++) {
        uint32_t s = (sel >> (4 * k)) & 7u;
        r |= (uint32_t)((x >> (8 * s)) & 0xffu) << (8 * k);
    }
    return r;
#endif
}

// rotate right by s (0..31)
BSG_HD uint32_t rotr(uint32_t x, uint32_t s)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_r(x, x, s);
#else
    s &= 31u;
    return s ? (x >> s) | (x << (32 - s)) : x;
#endif
}

BSG_HD uint32_t rotl(uint32_t x, uint32_t s)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_l(x, x, s);
#else
    s &= 31u;
    return s ? (x << s) | (x >> (32 - s)) : x;
#endif
}

// (hi:lo) >> s for s in 0..31, low word of the result
BSG_HD uint32_t funnel_r(uint32_t lo, uint32_t hi, uint32_t s)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_r(lo, hi, s);
#else
    s &= 31u;
    return s ? (lo >> s) | (hi << (32 - s)) : lo;
#endif
}

// ---------------------------------------------------------------------------
// 32 x 32 bit-matrix transpose held in 32 registers of one thread:
// afterwards a[r] bit e equals the old a[e] bit r.  The half and quarter
// block exchanges are byte permutes; the 4, 2 and 1 bit exchanges are masked
// swaps.
// ---------------------------------------------------------------------------
BSG_HD void transpose32(uint32_t (&a)[32])
{
#pragma unroll
    for (int k = 0; k < 16; k++) {
        uint32_t x = a[k], y = a[k + 16];
        a[k] = bperm(x, y, 0x5410);
        a[k + 16] = bperm(x, y, 0x7632);
    }
#pragma unroll
    for (int k = 0; k < 32; k++) {
        if (k & 8) continue;
        uint32_t x = a[k], y = a[k + 8];
        a[k] = bperm(x, y, 0x6240);
        a[k + 8] = bperm(x, y, 0x7351);
    }
#pragma unroll
    for (int k = 0; k < 32; k++) {
        if (k & 4) continue;
        uint32_t t = ((a[k] >> 4) ^ a[k + 4]) & 0x0f0f0f0fu;
        a[k + 4] ^= t;
        a[k] ^= t << 4;
    }
#pragma unroll
    for (int k = 0; k < 32; k++) {
        if (k & 2) continue;
        uint32_t t = ((a[k] >> 2) ^ a[k + 2]) & 0x33333333u;
        a[k + 2] ^= t;
        a[k] ^= t << 2;
    }
#pragma unroll
    for (int k = 0; k < 32; k++) {
        if (k & 1) continue;
        uint32_t t = ((a[k] >> 1) ^ a[k + 1]) & 0x55555555u;
        a[k + 1] ^= t;
        a[k] ^= t << 1;
    }
}

// ---------------------------------------------------------------------------
// Precision reduction of one float32 value (Sec. 3.2).
// q = 12 f s^2 as a float32.  When q is a positive normal float, the
// granularity exponent is k = max{k : 4^k < q}; from q's bits Q (biased
// exponent b, mantissa m) that is floor((b - 127 - [m == 0]) / 2), which
// equals ((Q + 0x7fffff) >> 24) - 64.  Adding 2^(k+23) to |x| (when |x| is
// smaller) leaves a float whose last place is 2^k, so the round-to-nearest-
// even addition rounds |x| to a multiple of 2^k with ties to the even
// multiple; subtracting 2^(k+23) again is exact.  |x| >= 2^(k+23) is already
// a multiple of 2^k; NaN and inf fail the comparison and pass through.
// ---------------------------------------------------------------------------
BSG_HD bool q_usable(uint32_t Q) { return (Q - 0x00800000u) < 0x7f000000u; }

BSG_HD uint32_t magic_bits(uint32_t Q)   // bit pattern of 2^(k+23)
{
    return (((Q + 0x007fffffu) >> 24) + 86u) << 23;
}

#ifdef __CUDACC__
BSG_D float round_to_granularity(float x, uint32_t Tbits)
{
    float T = __uint_as_float(Tbits);
    float ax = fabsf(x);
    float r = __fsub_rn(__fadd_rn(ax, T), T);
    return ax < T ? copysignf(r, x) : x;
}

BSG_D float reduce_one(float x, float q)
{
    uint32_t Q = __float_as_uint(q);
    return q_usable(Q) ? round_to_granularity(x, magic_bits(Q)) : x;
}
#endif

// Integer data: nearest multiple of 2^k, ties to the even multiple; k <= 0
// leaves x alone (a granularity of one or less); a nearest multiple above
// INT32_MAX is replaced by the lower one.  k is at most 63 here.
BSG_HD int32_t round_int_pow2(int32_t x, int k)
{
    if (k <= 0) return x;
    if (k >= 32) return 0;  // |x| <= 2^31 <= g / 2: the nearest (even) multiple is 0
    const int64_t g = (int64_t)1 << k;
    int64_t m = (int64_t)x >> k;  // floor
    const int64_t r = (int64_t)x - m * g, h = g >> 1;
    if (r > h || (r == h && (m & 1))) m++;
    int64_t y = m * g;
    if (y > INT32_MAX) y -= g;
    return (int32_t)y;
}

// Division by an invariant 32-bit divisor d >= 1 through a multiply-high:
// the unsigned method of T. Granlund and P. L. Montgomery, "Division by
// invariant integers using multiplication" (PLDI 1994, Sec. 4, Fig. 4.1).
// With l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (t + ((n - t) >> 1)) >> (l - 1) where t = mulhi(m, n); their
// Theorem 4.2 makes it exact for every 32-bit n.  d = 1 is kept apart
// (l - 1 would be negative).
struct FastDiv {
    uint32_t m, sh, d;
};

inline FastDiv fastdiv_init(uint32_t d)
{
    FastDiv f{0u, 0u, d};
    if (d <= 1) return f;
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) l++;
    f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
    f.sh = l - 1;
    return f;
}

BSG_HD uint32_t fastdiv(uint32_t n, const FastDiv &f)
{
    if (f.d == 1) return n;
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(f.m, n);
#else
    const uint32_t t = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
    return (t + ((n - t) >> 1)) >> f.sh;
}

// granularity exponent k = max{k : 4^k < q} from q's bits (see magic_bits)
BSG_HD int granularity_k(uint32_t Q) { return (int)((Q + 0x007fffffu) >> 24) - 64; }

#ifdef __CUDACC__
// Round one component given as its 32 bits: float32, or int32 when is_int.
BSG_D uint32_t reduce_bits(uint32_t xb, float q, bool is_int)
{
    const uint32_t Q = __float_as_uint(q);
    if (!q_usable(Q)) return xb;
    if (is_int) return (uint32_t)round_int_pow2((int32_t)xb, granularity_k(Q));
    return __float_as_uint(round_to_granularity(__uint_as_float(xb), magic_bits(Q)));
}
#endif

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier, bulk (TMA) copies, relaxed/acquire global accesses
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
BSG_D uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

BSG_D void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

BSG_D void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

BSG_D void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// the same for every state space (global memory written by the generic
// proxy, then read by a bulk copy)
BSG_D void fence_proxy_async_all()
{
    asm volatile("fence.proxy.async;" ::: "memory");
}

BSG_D void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy completing on `bar`; dst, src 16-byte aligned,
// bytes a multiple of 16
BSG_D void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// shared -> global bulk copy (bulk-group completion)
BSG_D void bulk_s2g(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}

BSG_D void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// wait until the committed bulk stores have finished reading shared memory
BSG_D void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// wait until the committed bulk stores are complete (visible in global memory)
BSG_D void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

BSG_D bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait on an mbarrier phase; false when the limit ran out
BSG_D bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < (1u << 22); it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

BSG_D uint64_t ld_relaxed_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

BSG_D void st_relaxed_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// record the first error in the status word (keeps the earliest nonzero code)
BSG_D void set_status(int *status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

BSG_D uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
#endif

}  // namespace bsg
