// CPU test of device code from paper_1503_00638_gb300/csrc: the register bit
// transposes and shuffles (per lane, plain host calls) and the warp LZ4
// encoder/decoder (on the warp emulator), checked against a naive bit loop
// and the oracle's LZ4 block codec.
#include "warp_emu.h"
#include "../../paper_1503_00638_gb300/csrc/lz4_warp.cuh"
#include "../../paper_1503_00638_gb300/csrc/shuffle.cuh"
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
extern "C" {
size_t orc_lz4_compress_block(const uint8_t *src, size_t n, uint8_t *dst, size_t cap);
int orc_lz4_decompress_block(const uint8_t *src, size_t src_len, uint8_t *dst, size_t dst_len);
int orc_bitshuffle(const void *vin, void *vout, size_t n, size_t es, size_t block_elems, int inverse);
int32_t orc_round_int(int32_t x, int k);
}
using namespace bsg;
alignas(16) static uint8_t A[70000], Bf[70000], C[70000], T[65536];
alignas(16) static uint8_t D2[70000];
alignas(16) static uint32_t FS[LZ4_FAST_SCRATCH / 4];

static int test_transpose(std::mt19937 &rng)
{
    int bad = 0;
    for (int it = 0; it < 2000; it++) {
        uint32_t a[32], b[32];
        for (int k = 0; k < 32; k++) a[k] = b[k] = (uint32_t)rng();
        transpose32(a);
        for (int r = 0; r < 32; r++)
            for (int e = 0; e < 32; e++) bad += ((a[r] >> e) & 1) != ((b[e] >> r) & 1);
    }
    return bad;
}

static int test_granularity_bits(std::mt19937 &rng)
{
    int bad = 0;
    for (int it = 0; it < 200000; it++) {
        uint32_t Q = (uint32_t)rng() & 0x7fffffffu;
        float q;
        memcpy(&q, &Q, 4);
        bool usable = q >= 1.17549435e-38f && std::isfinite(q);
        if (q_usable(Q) != usable) bad++;
        if (!usable) continue;
        int k = 0;
        while (ldexp(1.0, 2 * k) >= (double)q) k--;
        while (ldexp(1.0, 2 * (k + 1)) < (double)q) k++;
        uint32_t Tb = magic_bits(Q);
        float Tm;
        memcpy(&Tm, &Tb, 4);
        if ((double)Tm != ldexp(1.0, k + 23)) bad++;
        if (granularity_k(Q) != k) bad++;
    }
    return bad;
}

// multiply-high division against '/', over edge and random numerators
static int test_fastdiv(std::mt19937 &rng)
{
    int bad = 0;
    const uint32_t ds[] = {1, 2, 3, 5, 7, 16, 64, 136, 1000, 8256, 33024, 65535, 65536, 65537,
                           (1u << 31) - 1, 1u << 31, (1u << 31) + 1, 0xfffffffeu, 0xffffffffu};
    for (uint32_t d : ds) {
        const FastDiv f = fastdiv_init(d);
        const uint32_t ns[] = {0, 1, d - 1, d, d + 1, 2 * d - 1, 2 * d, 0x7fffffffu, 0x80000000u,
                               0xfffffffeu, 0xffffffffu};
        for (uint32_t n : ns) bad += fastdiv(n, f) != n / d;
        for (int it = 0; it < 20000; it++) {
            const uint32_t n = (uint32_t)rng();
            bad += fastdiv(n, f) != n / d;
        }
    }
    for (int it = 0; it < 20000; it++) {
        const uint32_t d = (uint32_t)rng() >> (rng() % 32);
        if (!d) continue;
        const FastDiv f = fastdiv_init(d);
        const uint32_t n = (uint32_t)rng();
        bad += fastdiv(n, f) != n / d;
    }
    return bad;
}

// integer rounding against the oracle's, over random and extreme values
static int test_round_int(std::mt19937 &rng)
{
    int bad = 0;
    const int32_t edge[] = {0, 1, -1, 2, -2, 3, -3, INT32_MAX, INT32_MIN, INT32_MAX - 1,
                            INT32_MIN + 1, 1 << 30, -(1 << 30), 12345, -12345};
    for (int k = -3; k <= 66; k++) {
        for (int32_t x : edge) bad += round_int_pow2(x, k) != orc_round_int(x, k);
        for (int it = 0; it < 4000; it++) {
            int32_t x = (int32_t)rng();
            if (it & 1) x >>= (rng() % 31);  // small magnitudes too
            bad += round_int_pow2(x, k) != orc_round_int(x, k);
            // ties: x = (2m + 1) 2^(k-1)
            if (k >= 1 && k <= 30) {
                int64_t m = (int32_t)rng() >> (k + 1);
                int64_t y = (2 * m + 1) * ((int64_t)1 << (k - 1));
                if (y >= INT32_MIN && y <= INT32_MAX)
                    bad += round_int_pow2((int32_t)y, k) != orc_round_int((int32_t)y, k);
            }
        }
    }
    return bad;
}

static int test_shuffles(std::mt19937 &rng)
{
    int bad = 0;
    for (int es : {1, 2, 4, 8})
        for (int B : {8, 24, 32, 64, 96, 1024, 2048, 8192}) {
            size_t S = (size_t)B * es;
            if (S > 65536) continue;
            for (size_t i = 0; i < S; i++) A[i] = (uint8_t)rng();
            for (uint32_t l = 0; l < 32; l++) shuffle_block(A, Bf, B, es, l);
            std::vector<uint8_t> ref(S);
            orc_bitshuffle(A, ref.data(), B, es, B, 0);
            bad += memcmp(Bf, ref.data(), S) != 0;
            for (uint32_t l = 0; l < 32; l++) unshuffle_block(Bf, C, B, es, l);
            bad += memcmp(A, C, S) != 0;
        }
    return bad;
}

static int g_inplace_cases = 0;

static int test_inplace_unshuffle(std::mt19937 &rng)
{
    int bad = 0;
    for (int es : {2, 4, 8})
        for (int B : {32, 64, 96, 128, 512, 1024, 1536, 2048, 3072, 4096}) {
            if (!unshuffle_inplace_ok(es, B)) continue;  // (B <= 1024 or 2048 for es 4)
            g_inplace_cases++;
            size_t S = (size_t)B * es;
            for (size_t i = 0; i < S; i++) A[i] = (uint8_t)rng();
            std::vector<uint8_t> rows(S);
            orc_bitshuffle(A, rows.data(), B, es, B, 0);
            memcpy(C, rows.data(), S);
            run_warp([&] {
                if (es == 2)
                    unshuffle2_inplace(C, B, threadIdx.x);
                else if (es == 4)
                    unshuffle4_inplace(C, B, threadIdx.x);
                else
                    unshuffle8_inplace(C, B, threadIdx.x);
            });
            bad += memcmp(A, C, S) != 0;
            if (shuffle_inplace_ok(es, B)) {
                memcpy(C, A, S);
                run_warp([&] {
                    if (es == 2)
                        shuffle2_inplace(C, B, threadIdx.x);
                    else if (es == 4)
                        shuffle4_inplace(C, B, threadIdx.x, [](uint32_t, uint32_t (&)[32]) {});
                    else
                        shuffle8_inplace(C, B, threadIdx.x);
                });
                bad += memcmp(rows.data(), C, S) != 0;
            }
        }
    // the transpose that also yields the encoder's equality bitmaps: bit-rows
    // with runs of equal words and words copied from the row above, the
    // bitmaps against lz4_eq_bitmaps on the rows it wrote
    for (int t = 0; t < 6; t++) {
        static uint32_t w[2048];
        for (int i = 0; i < 2048; i++) w[i] = (uint32_t)rng();
        for (int i = 1 + (int)(rng() % 7); i < 2040; i += 3 + (int)(rng() % 29)) {
            const int len = 1 + (int)(rng() % 6);
            for (int k = 0; k < len && i + k < 2048; k++)
                w[i + k] = (rng() & 1) ? w[i + k - 1] : (i + k >= 64 ? w[i + k - 64] : 0u);
        }
        if (t & 1)
            for (int i = 64 * (t + 3); i < 64 * (t + 5); i++) w[i] = 0;  // whole zero rows
        orc_bitshuffle(w, A, 2048, 4, 2048, 1);
        memcpy(C, A, 8192);
        uint32_t er[32][2], eu[32][2], fr[32][2], fu[32][2];
        run_warp([&] {
            uint32_t R2[2], U2[2];
            shuffle4_inplace_eq(C, threadIdx.x, [](uint32_t, uint32_t (&)[32]) {}, R2, U2);
            er[threadIdx.x][0] = R2[0], er[threadIdx.x][1] = R2[1];
            eu[threadIdx.x][0] = U2[0], eu[threadIdx.x][1] = U2[1];
        });
        bad += memcmp(C, w, 8192) != 0;
        run_warp([&] {
            uint32_t R2[2], U2[2];
            lz4_eq_bitmaps(reinterpret_cast<const uint32_t *>(C), 64, 64, threadIdx.x, R2, U2);
            fr[threadIdx.x][0] = R2[0], fr[threadIdx.x][1] = R2[1];
            fu[threadIdx.x][0] = U2[0], fu[threadIdx.x][1] = U2[1];
        });
        if (memcmp(er, fr, sizeof er) || memcmp(eu, fu, sizeof eu)) {
            fprintf(stderr, "fused equality bitmaps differ (case %d)\n", t);
            bad++;
        }
    }
    return bad;
}

// In-place decoding of blocks over 8 KiB as decompress_inplace_any_kernel
// lays them out: a buffer of S + 2 S / 255 + 160 bytes (rounded up to 16; the
// kernel's inplace_any_buf), the stream's image 32 bytes before its end at
// each 16-byte phase, oracle streams of incompressible, compressible and
// mixed blocks (a long literal run after compressible data stresses the
// margin most).
static int test_inplace_large(std::mt19937 &rng)
{
    int bad = 0;
    static uint8_t IB[66208 + 64];
    for (uint32_t S : {16384u, 32768u, 65536u}) {
        const uint32_t E = (S + 2u * S / 255u + 160u + 15u) & ~15u;
        for (int kind = 0; kind < 4; kind++) {
            std::vector<uint8_t> m(S);
            for (uint32_t i = 0; i < S; i++) {
                const uint8_t r = (uint8_t)rng();
                m[i] = kind == 0 ? r                                    // incompressible
                     : kind == 1 ? (uint8_t)((i / 300) & 3)             // long matches
                     : kind == 2 ? (i < S / 2 ? 0 : r)                  // zeros, then noise
                                 : ((i / 97) % 3 == 0 ? r : (uint8_t)(i / 1000));
            }
            std::vector<uint8_t> oc(lz4_bound(S) + 16);
            const uint32_t cs = (uint32_t)orc_lz4_compress_block(m.data(), S, oc.data(), oc.size());
            for (uint32_t ph : {0u, 7u, 15u}) {
                const uint32_t len = cs + 4, off = (E - len - 32u) & ~15u;
                memset(IB, 0x5A, sizeof IB);
                memcpy(IB + off + ph + 4, oc.data(), cs);
                int rc = -1;
                run_warp([&] {
                    int r = lz4_decode_warp(IB + off, ph + 4, cs, IB, S);
                    if (threadIdx.x == 0) rc = r;
                });
                if (rc || memcmp(IB, m.data(), S)) {
                    fprintf(stderr, "large in-place decode differs S=%u kind=%d phase=%u rc=%d\n", S,
                            kind, ph, rc);
                    bad++;
                }
            }
        }
    }
    return bad;
}

static int test_lz4(std::mt19937 &rng, int level, double &gpu_ratio, double &orc_ratio)
{
    int bad = 0;
    std::vector<std::vector<uint8_t>> cases;
    std::vector<uint32_t> rows;
    for (int S : {0, 1, 12, 13, 17, 100, 8192}) {
        std::vector<uint8_t> z(S, 0), r(S), m(S);
        for (auto &x : r) x = (uint8_t)rng();
        for (int i = 0; i < S; i++) m[i] = (i / 37) % 3 == 0 ? (uint8_t)rng() : (uint8_t)((i / 100) & 7);
        for (auto *c : {&z, &r, &m}) {
            cases.push_back(*c);
            rows.push_back((uint32_t)(S / 32));
        }
    }
    // short low-entropy blocks: matches near the end-of-block limits
    for (int t = 0; t < 150; t++) {
        int S = 13 + (int)(rng() % 120);
        std::vector<uint8_t> m(S);
        int alpha = 1 + (int)(rng() % 3);
        for (auto &x : m) x = (uint8_t)(rng() % alpha);
        cases.push_back(m);
        rows.push_back((uint32_t)(4 * (rng() % 8)));
    }
    for (int t = 0; t < 16; t++) {
        int S = 128 * (1 + (int)(rng() % 64));
        std::vector<uint8_t> m(S);
        int alpha = 1 + (int)(rng() % 3);
        for (int i = 0; i < S; i++) m[i] = (i / (1 + rng() % 97)) % 5 == 0 ? (uint8_t)rng() : (uint8_t)(rng() % alpha);
        cases.push_back(m);
        rows.push_back((uint32_t)(S / 32));
    }
    for (int t = 0; t < 4; t++) {
        std::vector<int32_t> w(2048);
        int32_t x = 0;
        for (auto &v : w) {
            x += (rng() & 1 ? 1 : -1) * (1 << (rng() % 7));
            v = x;
        }
        std::vector<uint8_t> sh(8192);
        orc_bitshuffle(w.data(), sh.data(), 2048, 4, 2048, 0);
        cases.push_back(sh);
        rows.push_back(256);
    }
    for (int t = 0; t < 4; t++) {
        std::vector<uint16_t> w(4096);
        int32_t x = 0;
        for (auto &v : w) {
            x += (rng() & 1 ? 1 : -1) * (1 << (rng() % 7));
            v = (uint16_t)x;
        }
        std::vector<uint8_t> sh(8192);
        orc_bitshuffle(w.data(), sh.data(), 4096, 2, 4096, 0);
        cases.push_back(sh);
        rows.push_back(512);
    }
    // blocks made of stretches of zero words, repeated words, copies of the
    // bit-row above, random words and mixtures, with lengths that start and
    // end anywhere relative to the 256-byte segments of the fast encoder's
    // lanes (matches spilling into the next segments, row and run candidates
    // side by side at segment starts)
    for (int t = 0; t < 48; t++) {
        const int S = t < 32 ? 8192 : 128 * (1 + (int)(rng() % 64));
        const uint32_t rl = t % 3 == 0 ? 256u : 4u * (uint32_t)(1 + rng() % 64);
        std::vector<uint32_t> w(S / 4);
        size_t i = 0;
        while (i < w.size()) {
            const int kind = (int)(rng() % 6);
            size_t len = 1 + rng() % (rng() % 4 == 0 ? 700 : 40);
            for (size_t k = 0; k < len && i < w.size(); k++, i++) {
                const uint32_t r = (uint32_t)rng();
                switch (kind) {
                case 0: w[i] = 0; break;
                case 1: w[i] = i ? w[i - 1] : r; break;
                case 2: w[i] = i >= rl / 4 ? w[i - rl / 4] : r; break;
                case 3: w[i] = r; break;
                case 4: w[i] = (k % 5 == 4) ? r : (i ? w[i - 1] : 0); break;
                default: w[i] = (i >= rl / 4 && k % 3) ? w[i - rl / 4] ^ (r & 0x01000000u) : r; break;
                }
            }
        }
        std::vector<uint8_t> m(S);
        memcpy(m.data(), w.data(), S);
        cases.push_back(m);
        rows.push_back(rl);
    }
    size_t tg = 0, to = 0, tin = 0;
    for (size_t ci = 0; ci < cases.size(); ci++) {
        auto &c = cases[ci];
        uint32_t S = (uint32_t)c.size();
        memset(A, 0xEE, S + 64);
        memcpy(A, c.data(), S);
        uint32_t cs = 0;
        run_warp([&] {
            uint32_t o = level ? lz4_encode_warp<1, 11>(A, S, rows[ci], Bf, (uint16_t *)T)
                               : lz4_encode_warp<0, 11>(A, S, rows[ci], Bf, (uint16_t *)T);
            if (threadIdx.x == 0) cs = o;
        });
        if (cs > lz4_bound(S)) { bad++; continue; }
        if (level == 0 && S % 4 == 0) {
            // the bitmap-driven encoder follows the same parse rule
            uint32_t cs2 = 0;
            static uint8_t E[70000];
            memset(E, 0xCD, S + 64);
            run_warp([&] {
                uint32_t o = lz4_encode_bitmap(A, S, rows[ci], E, (uint32_t *)T);
                if (threadIdx.x == 0) cs2 = o;
            });
            if (cs2 != cs || memcmp(E, Bf, cs)) {
                fprintf(stderr, "bitmap encoder differs S=%u rows=%u %u vs %u\n", S, rows[ci], cs2, cs);
                bad++;
            }
            if (S % 128 == 0 && S <= 8192 && S > 0) {
                uint32_t cs3 = 0;
                memset(E, 0xCD, S + 64);
                run_warp([&] {
                    uint32_t o = lz4_encode_bitmap_fast(A, S, rows[ci], E, FS);
                    if (threadIdx.x == 0) cs3 = o;
                });
                if (cs3 != cs || memcmp(E, Bf, cs)) {
                    fprintf(stderr, "fast bitmap encoder differs S=%u rows=%u %u vs %u\n", S, rows[ci], cs3, cs);
                    bad++;
                }
                // a node table of 8 entries: most blocks take the candidate walk
                // (every other case, to keep the emulation's run time down)
                if (ci % 2 == 0) {
                    memset(E, 0xCD, S + 64);
                    run_warp([&] {
                        uint32_t o = lz4_encode_bitmap_fast<8>(A, S, rows[ci], E, FS);
                        if (threadIdx.x == 0) cs3 = o;
                    });
                    if (cs3 != cs || memcmp(E, Bf, cs)) {
                        fprintf(stderr, "fast bitmap encoder (walk) differs S=%u rows=%u %u vs %u\n", S,
                                rows[ci], cs3, cs);
                        bad++;
                    }
                }
            }
        }
        std::vector<uint8_t> out(S + 1);
        if (orc_lz4_decompress_block(Bf, cs, out.data(), S) || memcmp(out.data(), c.data(), S)) bad++;
        int rc = -1;
        // decode from every alignment of the stream start, as the kernel does
        for (uint32_t sh = 0; sh < 4 && !bad; sh++) {
            memset(D2, 0, cs + 32);
            memcpy(D2 + sh, Bf, cs);
            run_warp([&] {
                int r = lz4_decode_warp(D2, sh, cs, C, S);
                if (threadIdx.x == 0) rc = r;
            });
            if (rc || memcmp(C, c.data(), S)) bad++;
        }
        // in-place decoding as decompress_inplace_kernel does it: the stream
        // (after its 4-byte length field) at the end of an 8352-byte buffer
        for (uint32_t ph = 0; ph < 16 && !bad && S <= 8192; ph += 13) {
            static uint8_t IB[8352 + 64];
            const uint32_t len = cs + 4, off = (8352u - len - 32u) & ~15u;
            memset(IB, 0x5A, sizeof IB);
            memcpy(IB + off + ph + 4, Bf, cs);
            run_warp([&] {
                int r = lz4_decode_warp(IB + off, ph + 4, cs, IB, S);
                if (threadIdx.x == 0) rc = r;
            });
            if (rc || memcmp(IB, c.data(), S)) {
                fprintf(stderr, "in-place decode differs S=%u cs=%u phase=%u rc=%d\n", S, cs, ph, rc);
                bad++;
            }
        }
        std::vector<uint8_t> oc(lz4_bound(S) + 16);
        size_t ocs = orc_lz4_compress_block(c.data(), S, oc.data(), oc.size());
        for (uint32_t ph = 7; ph < 16 && !bad && S <= 8192; ph += 16) {
            static uint8_t IB2[8352 + 64];
            const uint32_t len = (uint32_t)ocs + 4, off = (8352u - len - 32u) & ~15u;
            memset(IB2, 0x5A, sizeof IB2);
            memcpy(IB2 + off + ph + 4, oc.data(), ocs);
            run_warp([&] {
                int r = lz4_decode_warp(IB2 + off, ph + 4, (uint32_t)ocs, IB2, S);
                if (threadIdx.x == 0) rc = r;
            });
            if (rc || memcmp(IB2, c.data(), S)) {
                fprintf(stderr, "in-place decode (oracle stream) differs S=%u cs=%zu phase=%u rc=%d\n", S, ocs, ph, rc);
                bad++;
            }
        }
        memset(D2, 0, ocs + 16);
        memcpy(D2 + 3, oc.data(), ocs);
        run_warp([&] {
            int r = lz4_decode_warp(D2, 3, (uint32_t)ocs, C, S);
            if (threadIdx.x == 0) rc = r;
        });
        if (rc || memcmp(C, c.data(), S)) bad++;
        tg += cs;
        to += ocs;
        tin += S;
    }
    gpu_ratio = (double)tg / tin;
    orc_ratio = (double)to / tin;
    return bad;
}

int main()
{
    std::mt19937 rng(7);
    int t = test_transpose(rng), g = test_granularity_bits(rng), s = test_shuffles(rng);
    g += test_round_int(rng);
    g += test_fastdiv(rng);
    s += test_inplace_unshuffle(rng);
    printf("in-place shapes %d\n", g_inplace_cases);
    if (g_inplace_cases != 20) s++;  // es 2: 7 shapes, es 4: 7, es 8: 6
    double gr0 = 0, gr1 = 0, orr = 0;
    int l0 = test_lz4(rng, 0, gr0, orr);
    int l1 = test_lz4(rng, 1, gr1, orr);
    l0 += test_inplace_large(rng);
    printf("transpose %d granularity %d shuffle %d lz4 %d %d ratio level0 %.4f level1 %.4f "
           "oracle %.4f\n", t, g, s, l0, l1, gr0, gr1, orr);
    return (t || g || s || l0 || l1) ? 1 : 0;
}
