// Warp-cooperative LZ4 block encoder and decoder on shared memory (Sec. 4.1:
// an LZ77-class code of literal runs and (offset, length) back-references,
// run-length encoding when the length exceeds the offset; Sec. 4.2.1: one
// block at a time while it is on chip).
//
// Block format (the public LZ4 block format): each sequence is a token
// (literal length in the high nibble, match length - 4 in the low nibble,
// 15 = more length bytes follow, each 255 continuing), the literals, a 2-byte
// little-endian offset and the match-length bytes; the last sequence is
// literals only; the last 5 bytes of a block are literals and the last
// match starts at least 12 bytes before the end.
#pragma once

#include "common.cuh"

namespace bsg {

constexpr uint32_t LZ4_MINMATCH = 4;
constexpr uint32_t LZ4_LASTLITERALS = 5;
constexpr uint32_t LZ4_MFLIMIT = 12;

BSG_HD uint32_t lz4_bound(uint32_t n) { return n + n / 255u + 16u; }

// Failed probe windows after which the probe stride doubles (4 -> 8 -> 16
// bytes): skips quickly through incompressible bit rows.
constexpr uint32_t LZ4_ACCEL_WINDOWS = 4;

// Shortest match the GPU encoders emit (the format allows 4): two words at
// level 1, three at level 0.  A short match saves a few bytes but costs a
// whole sequence, and the number of sequences bounds both the level-0 parse
// and the decoder; matches of two words are a third of the level-0 sequences
// of bitshuffled visibilities but carry about 2 % of the matched bytes.
constexpr uint32_t LZ4_GPU_MINMATCH = 8;
constexpr uint32_t LZ4_L0_MINWORDS = 3;
constexpr uint32_t LZ4_L0_MINMATCH = 4 * LZ4_L0_MINWORDS;
template <int LEVEL>
constexpr uint32_t LZ4_MINMATCH_OF = LEVEL >= 1 ? LZ4_GPU_MINMATCH : LZ4_L0_MINMATCH;

#if defined(__CUDACC__) || defined(BSG_WARP_EMU)

// 4 bytes starting at byte q of a word-aligned shared buffer (little endian);
// reads the aligned words at q & ~3 and the next one
BSG_D uint32_t ld32u(const uint8_t *base, uint32_t q)
{
#ifdef BSG_WARP_EMU
    emu_check_aligned4(base);
#endif
    const uint32_t *w = reinterpret_cast<const uint32_t *>(base);
    uint32_t i = q >> 2;
    return funnel_r(w[i], w[i + 1], (q & 3u) * 8u);
}

// Warp copy of len bytes src[s..] -> dst[d..] (word-aligned shared buffers,
// the ranges must not overlap): bytes up to dst's next word boundary, whole
// words assembled by funnel shifts, then the ragged end.  src is read up to
// 7 bytes past s + len.
BSG_D void warp_copy(uint8_t *dst, uint32_t d, const uint8_t *src, uint32_t s, uint32_t len,
                     uint32_t lane)
{
#ifdef BSG_WARP_EMU
    emu_check_aligned4(dst);
    emu_check_aligned4(src);
#endif
    if (len <= 32) {
        if (lane < len) dst[d + lane] = src[s + lane];
        return;
    }
    const uint32_t a0 = (d + 3u) & ~3u, a1 = (d + len) & ~3u;
    const uint32_t head = a0 - d, tail = d + len - a1;
    if (lane < head) dst[d + lane] = src[s + lane];
    if (lane >= 28 && lane - 28 < tail) dst[a1 + lane - 28] = src[s + (a1 - d) + lane - 28];
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    if (((d - s) & 3u) == 0) {
        // source and destination share their word alignment: plain word copy
        const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
        const int sh = (int)(s - d) / 4;  // signed word distance (exact: a multiple of 4)
        for (uint32_t w = (a0 >> 2) + lane; w < (a1 >> 2); w += 32) d32[w] = s32[(int)w + sh];
        return;
    }
    for (uint32_t w = (a0 >> 2) + lane; w < (a1 >> 2); w += 32) d32[w] = ld32u(src, s + 4 * w - d);
}

// Copy of up to 32 independent byte ranges, range k (k < n) held by lane k as
// (source offset a, destination offset d, length len).  Ranges of at most
// LZ4_RANGE_SHORT bytes go four at a time, eight lanes each (head bytes up to
// dst's word boundary, whole words from funnel-shifted loads, ragged end), so
// that short runs do not each cost a whole-warp pass; longer ones go one
// after another with the whole warp, so that a long run does not keep 24
// lanes idle.  The ranges must not overlap each other or the sources.
constexpr uint32_t LZ4_RANGE_SHORT = 64;

BSG_D void warp_copy_ranges(uint8_t *dst, const uint8_t *src, uint32_t n, uint32_t a, uint32_t d,
                            uint32_t len, uint32_t lane)
{
#ifdef BSG_WARP_EMU
    emu_check_aligned4(dst);
    emu_check_aligned4(src);
#endif
    const uint32_t g = lane >> 3, sl = lane & 7u;
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t base = 0; base < n; base += 4) {
        const uint32_t k = base + g;
        const uint32_t ak = __shfl_sync(FULL, a, k & 31u), dk = __shfl_sync(FULL, d, k & 31u);
        const uint32_t lk0 = __shfl_sync(FULL, len, k & 31u);
        const uint32_t lk = k < n && lk0 <= LZ4_RANGE_SHORT ? lk0 : 0u;
        if (lk == 0) continue;
        if (lk <= 8) {
            if (sl < lk) dst[dk + sl] = src[ak + sl];
            continue;
        }
        const uint32_t a0 = (dk + 3u) & ~3u, a1 = (dk + lk) & ~3u;
        const uint32_t head = a0 - dk, tail = dk + lk - a1;
        if (sl < head) dst[dk + sl] = src[ak + sl];
        if (sl >= 4 && sl - 4 < tail) dst[a1 + sl - 4] = src[ak + (a1 - dk) + sl - 4];
        for (uint32_t w = (a0 >> 2) + sl; w < (a1 >> 2); w += 8) d32[w] = ld32u(src, ak + 4 * w - dk);
    }
    uint32_t longs = __ballot_sync(FULL, lane < n && len > LZ4_RANGE_SHORT);
    while (longs) {
        const uint32_t k = (uint32_t)(__ffs(longs) - 1);
        longs &= longs - 1;
        const uint32_t ak = __shfl_sync(FULL, a, k), dk = __shfl_sync(FULL, d, k);
        const uint32_t lk = __shfl_sync(FULL, len, k);
        const uint32_t a0 = (dk + 3u) & ~3u, a1 = (dk + lk) & ~3u;
        const uint32_t head = a0 - dk, tail = dk + lk - a1;
        if (lane < head) dst[dk + lane] = src[ak + lane];
        if (lane >= 4 && lane - 4 < tail) dst[a1 + lane - 4] = src[ak + (a1 - dk) + lane - 4];
        const uint32_t q = ak - dk;  // source byte of destination byte 0 (mod 2^32)
        for (uint32_t w = (a0 >> 2) + lane; w < (a1 >> 2); w += 32) d32[w] = ld32u(src, q + 4 * w);
    }
}

// Forward copy for a decoder that may write over its own input (in-place
// decoding, the unread input starting at or after the write position): every
// byte of a step is loaded before any lane stores that step, so no lane, however
// far ahead, overwrites input another lane has still to read.  Head and tail
// bytes are loaded up front, the head stored first, the tail last.
BSG_D void warp_copy_ordered(uint8_t *dst, uint32_t d, const uint8_t *src, uint32_t s,
                             uint32_t len, uint32_t lane)
{
#ifdef BSG_WARP_EMU
    emu_check_aligned4(dst);
    emu_check_aligned4(src);
#endif
    if (len <= 32) {
        const uint8_t v = lane < len ? src[s + lane] : 0;
        __syncwarp();
        if (lane < len) dst[d + lane] = v;
        return;
    }
    const uint32_t a0 = (d + 3u) & ~3u, a1 = (d + len) & ~3u;
    const uint32_t head = a0 - d, tail = d + len - a1;
    const bool ht = lane >= 28 && lane - 28 < tail;
    const uint8_t hv = lane < head ? src[s + lane] : 0;
    const uint8_t tv = ht ? src[s + (a1 - d) + lane - 28] : 0;
    __syncwarp();
    if (lane < head) dst[d + lane] = hv;
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    const uint32_t w1 = a1 >> 2;
    for (uint32_t base = a0 >> 2; base < w1; base += 32) {
        const uint32_t w = base + lane;
        const uint32_t v = w < w1 ? ld32u(src, s + 4 * w - d) : 0u;
        __syncwarp();
        if (w < w1) d32[w] = v;
    }
    __syncwarp();
    if (ht) dst[a1 + lane - 28] = tv;
}

// Warp fill of len bytes at dst[d..] with the byte b.
BSG_D void warp_fill(uint8_t *dst, uint32_t d, uint32_t b, uint32_t len, uint32_t lane)
{
#ifdef BSG_WARP_EMU
    emu_check_aligned4(dst);
#endif
    if (len <= 32) {
        if (lane < len) dst[d + lane] = (uint8_t)b;
        return;
    }
    const uint32_t a0 = (d + 3u) & ~3u, a1 = (d + len) & ~3u;
    const uint32_t head = a0 - d, tail = d + len - a1;
    if (lane < head) dst[d + lane] = (uint8_t)b;
    if (lane >= 28 && lane - 28 < tail) dst[a1 + lane - 28] = (uint8_t)b;
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    const uint32_t v = b * 0x01010101u;
    for (uint32_t w = (a0 >> 2) + lane; w < (a1 >> 2); w += 32) d32[w] = v;
}

// Warp fill of len bytes at dst[d..] repeating the off bytes before d, for
// off in {1, 2, 4} (so the pattern repeats within every aligned word).
BSG_D void warp_fill_pattern(uint8_t *dst, uint32_t d, uint32_t off, uint32_t len, uint32_t lane)
{
#ifdef BSG_WARP_EMU
    emu_check_aligned4(dst);
#endif
    // byte i of the output is dst[d - off + i % off]
    if (len <= 32) {
        const uint8_t v = dst[d - off + (lane & (off - 1))];
        __syncwarp();
        if (lane < len) dst[d + lane] = v;
        return;
    }
    const uint32_t a0 = (d + 3u) & ~3u, a1 = (d + len) & ~3u;
    const uint32_t head = a0 - d, tail = d + len - a1;
    // the aligned word at a0 starts with output byte (a0 - d), i.e. pattern
    // byte (a0 - d) % off; the word is the same at every aligned address
    uint32_t word = 0;
#pragma unroll
    for (uint32_t k = 0; k < 4; k++) word |= (uint32_t)dst[d - off + ((head + k) & (off - 1))] << (8 * k);
    uint8_t hv = 0, tv = 0;
    if (lane < head) hv = dst[d - off + (lane & (off - 1))];
    if (lane >= 28 && lane - 28 < tail) tv = dst[d - off + ((a1 - d + lane - 28) & (off - 1))];
    __syncwarp();
    if (lane < head) dst[d + lane] = hv;
    if (lane >= 28 && lane - 28 < tail) dst[a1 + lane - 28] = tv;
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t w = (a0 >> 2) + lane; w < (a1 >> 2); w += 32) d32[w] = word;
}

// Length bytes of an LZ4 field: v >= 15 is 15 in the nibble, then
// (v - 15) / 255 bytes of 255 and one byte of (v - 15) % 255.
BSG_D uint32_t lz4_ext_count(uint32_t v) { return v >= 15 ? (v - 15) / 255 + 1 : 0; }

BSG_D void lz4_put_ext(uint8_t *dst, uint32_t o, uint32_t v, uint32_t n, uint32_t lane)
{
    for (uint32_t k = lane; k < n; k += 32) dst[o + k] = k + 1 < n ? 255u : (uint8_t)((v - 15) % 255u);
}

// Write one sequence (literals [anchor, mp), match of `len` bytes at
// distance `off`) at dst[o..]; returns the new output length.
BSG_D uint32_t lz4_emit(uint8_t *dst, uint32_t o, const uint8_t *src, uint32_t anchor,
                        uint32_t mp, uint32_t off, uint32_t len, uint32_t lane)
{
    const uint32_t LL = mp - anchor;
    const uint32_t ML = len - LZ4_MINMATCH;
    const uint32_t nll = lz4_ext_count(LL), nml = lz4_ext_count(ML);
    if (lane == 0) dst[o] = (uint8_t)(((LL < 15 ? LL : 15) << 4) | (ML < 15 ? ML : 15));
    lz4_put_ext(dst, o + 1, LL, nll, lane);
    const uint32_t lo = o + 1 + nll;
    warp_copy(dst, lo, src, anchor, LL, lane);
    const uint32_t oo = lo + LL;
    if (lane == 1) dst[oo] = (uint8_t)(off & 255u);
    if (lane == 2) dst[oo + 1] = (uint8_t)(off >> 8);
    lz4_put_ext(dst, oo + 2, ML, nml, lane);
    return oo + 2 + nml;
}

// Literals-only last sequence [anchor, S).
BSG_D uint32_t lz4_emit_last(uint8_t *dst, uint32_t o, const uint8_t *src, uint32_t anchor,
                             uint32_t S, uint32_t lane)
{
    const uint32_t LL = S - anchor;
    const uint32_t nll = lz4_ext_count(LL);
    if (lane == 0) dst[o] = (uint8_t)((LL < 15 ? LL : 15) << 4);
    lz4_put_ext(dst, o + 1, LL, nll, lane);
    warp_copy(dst, o + 1 + nll, src, anchor, LL, lane);
    return o + 1 + nll + LL;
}

// Encode src[0, S) (word aligned, readable up to S + 8) into dst (capacity
// lz4_bound(S)), taking only matches of at least LZ4_MINMATCH_OF<LEVEL>
// bytes.
//
// Each step probes 32 word-aligned positions p at once.  Candidates:
//  * the same column of the previous bit-row, p - rowlen (a bit-row repeating
//    the one before it, as the most significant rows of two's-complement or
//    sign/exponent data do, Sec. 4.2); rowlen = 0 disables it;
//  * p - 4, a run (all-zero rows of the bits rounded away, Sec. 3.2);
//  * LEVEL >= 1 only: the last probed position with the same 4-byte hash
//    (nearest earlier lane of this step, else a 16-bit table entry written by
//    the highest lane of each hash group, so nothing depends on scheduling);
//    after LZ4_ACCEL_WINDOWS fruitless steps the probe stride doubles (to 16
//    bytes at most).
// The first position whose candidate agrees on the minimum match is taken,
// extended back by up to 3 bytes and forward warp-wide.  Returns the compressed size,
// or 0xffffffff if the progress guard tripped (cannot happen for valid sizes).
template <int LEVEL, int HBITS>
BSG_D uint32_t lz4_encode_warp(const uint8_t *src, uint32_t S, uint32_t rowlen, uint8_t *dst,
                               uint16_t *table)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt = lanemask_lt();
    const uint32_t le = lt | (1u << lane);
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    if (LEVEL >= 1) {
        uint4 *t4 = reinterpret_cast<uint4 *>(table);
        for (uint32_t i = lane; i < (2u << HBITS) / 16u; i += 32) t4[i] = make_uint4(0, 0, 0, 0);
        __syncwarp();
    }
    if (rowlen & 3u) rowlen = 0;
    uint32_t anchor = 0, o = 0;
    if (S >= LZ4_MFLIMIT + 1 && S >= LZ4_LASTLITERALS + LZ4_MINMATCH_OF<LEVEL>) {
        // a probe at p verifies MM bytes, so it must end by the match-end
        // bound (p + MM <= S - 5), which is also below the last allowed match start
        constexpr uint32_t MM = LZ4_MINMATCH_OF<LEVEL>;
        const uint32_t mflimit = S - LZ4_LASTLITERALS - MM;
        const uint32_t matchlimit = S - LZ4_LASTLITERALS;  // match end bound
        uint32_t pos = 0, fails = 0;
        const uint32_t guard = S / 4 + 8;
        uint32_t it = 0;
        while (pos <= mflimit) {
            if (++it > guard) return 0xffffffffu;
            uint32_t step = 4;
            if (LEVEL >= 1) {
                const uint32_t sh = fails / LZ4_ACCEL_WINDOWS;
                step = 4u << (sh < 2 ? sh : 2);
            }
            const uint32_t p = pos + step * lane;
            const bool valid = p <= mflimit;
            const uint32_t wi = p >> 2;
            const uint32_t w0 = valid ? s32[wi] : 0u;
            const uint32_t w1 = valid ? s32[wi + 1] : 0u;
            static_assert(MM == 8 || MM == 12, "probes verify two or three words");
            const uint32_t w2 = (MM > 8 && valid) ? s32[wi + 2] : 0u;
            uint32_t off = 0;
            if (valid && rowlen && p >= rowlen) {
                const uint32_t ri = (p - rowlen) >> 2;
                if (s32[ri] == w0 && s32[ri + 1] == w1 && (MM <= 8 || s32[ri + 2] == w2))
                    off = rowlen;
            }
            if (valid && off == 0 && p >= 4 && w1 == w0 && (MM <= 8 || w2 == w0) &&
                s32[wi - 1] == w0)
                off = 4;
            if (LEVEL >= 1) {
                const uint32_t h = (w0 * 2654435761u) >> (32 - HBITS);
                const uint32_t grp = __match_any_sync(FULL, valid ? h : 0x80000000u);
                const uint32_t lower = grp & lt;
                int32_t cand = valid ? (int32_t)table[h] * 4 - 4 : -1;
                if (valid && lower) cand = (int32_t)(pos + step * (31 - __clz(lower)));
                if (valid && off == 0 && cand >= 0 && s32[cand >> 2] == w0 &&
                    s32[(cand >> 2) + 1] == w1)
                    off = p - (uint32_t)cand;
                const uint32_t mm0 = __ballot_sync(FULL, off != 0);
                const uint32_t vm = __ballot_sync(FULL, valid);
                // insert the probed positions up to the match (all of them if none)
                const uint32_t upto = mm0 ? ((2u << (__ffs(mm0) - 1)) - 1u) : FULL;
                const uint32_t mine = grp & upto & vm;
                if (valid && (upto >> lane & 1u) && (mine & ~le) == 0)
                    table[h] = (uint16_t)((p >> 2) + 1);
                __syncwarp();
            }
            const uint32_t mm = __ballot_sync(FULL, off != 0);
            if (mm == 0) {
                fails++;
                pos += step * 32;
                continue;
            }
            const uint32_t fl = __ffs(mm) - 1;
            const uint32_t p0 = pos + step * fl;
            const uint32_t moff = __shfl_sync(FULL, off, fl);
            uint32_t mp = p0;
            // back up over up to 3 equal bytes (never before the literal anchor)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (mp > anchor && mp > moff && src[mp - 1] == src[mp - 1 - moff]) mp--;
            }
            const uint32_t mc = mp - moff;
            uint32_t len = p0 + MM - mp;   // the verified bytes, and the backed-up ones
            // extend forward, 128 bytes per step
            for (uint32_t g2 = 0; g2 < S; g2 += 128) {
                const uint32_t q = mp + len + 4 * lane;
                const int room = (int)matchlimit - (int)q;
                uint32_t eq = 0;
                if (room > 0) {
                    const uint32_t x = ld32u(src, q) ^ ld32u(src, mc + len + 4 * lane);
                    eq = x ? ((uint32_t)(__ffs(x) - 1) >> 3) : 4u;
                    if ((int)eq > room) eq = (uint32_t)room;
                }
                const uint32_t stop = __ballot_sync(FULL, eq < 4);
                if (stop == 0) {
                    len += 128;
                    continue;
                }
                const uint32_t sl = __ffs(stop) - 1;
                len += 4 * sl + __shfl_sync(FULL, eq, sl);
                break;
            }
            o = lz4_emit(dst, o, src, anchor, mp, moff, len, lane);
            anchor = mp + len;
            pos = (anchor + 3u) & ~3u;
            fails = 0;
        }
    }
    o = lz4_emit_last(dst, o, src, anchor, S, lane);
    __syncwarp();
    return o;
}

// Smallest word index w >= start with bit w of the bitmap E clear, or cap if
// none is below cap.  E has a clear bit at or before every index it covers.
BSG_D uint32_t bitmap_first_zero(const uint32_t *E, uint32_t start, uint32_t cap, uint32_t lane)
{
    if (start >= cap) return cap;
    for (uint32_t qb = start >> 5; qb * 32 < cap; qb += 32) {
        const uint32_t q = qb + lane;
        uint32_t z = 0;
        if (q * 32 < cap) {
            z = ~E[q];
            if (q == (start >> 5)) z &= ~0u << (start & 31u);
        }
        const uint32_t m = __ballot_sync(FULL, z != 0);
        if (m) {
            const uint32_t fl = __ffs(m) - 1;
            const uint32_t zz = __shfl_sync(FULL, z, fl);
            const uint32_t w = (qb + fl) * 32 + (__ffs(zz) - 1);
            return w < cap ? w : cap;
        }
    }
    return cap;
}

// Level-0 encoder (same parse rule as lz4_encode_warp<0>: matches of at least
// LZ4_L0_MINMATCH bytes at word-aligned positions against the previous bit-row
// or the previous word, extended back up to 3 bytes and forward), driven by
// two word-equality bitmaps built in one parallel pass:
//   Erow bit w: word w equals word w - rowlen/4;  Erun bit w: word w equals w - 1.
// A candidate at word w needs bits w .. w + LZ4_L0_MINWORDS - 1; a match then covers
// every following word whose bit is set, plus the equal leading bytes of the
// first word that differs.  The serial part of the parse is a handful of
// bitmap scans per sequence instead of a probe loop.  S must be a multiple of
// 4; bm holds 2 * (S/128 + 2) words of shared scratch.
BSG_D uint32_t lz4_encode_bitmap(const uint8_t *src, uint32_t S, uint32_t rowlen, uint8_t *dst,
                                 uint32_t *bm)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    const uint32_t NW = S / 4;
    const uint32_t NB = (NW + 31) / 32;
    const uint32_t R = (rowlen & 3u) ? 0u : rowlen / 4;
    uint32_t *Erow = bm, *Erun = bm + NB + 1;
    for (uint32_t b = 0; b < NB; b++) {
        const uint32_t w = 32 * b + lane;
        const bool in = w < NW;
        const uint32_t x = in ? s32[w] : 0u;
        uint32_t xp = __shfl_up_sync(FULL, x, 1);
        if (lane == 0) xp = w >= 1 ? s32[w - 1] : ~x;
        const uint32_t xr = (in && R && w >= R) ? s32[w - R] : ~x;
        const uint32_t row = __ballot_sync(FULL, in && R && w >= R && x == xr);
        const uint32_t run = __ballot_sync(FULL, in && w >= 1 && x == xp);
        if (lane == 0) {
            Erow[b] = row;
            Erun[b] = run;
        }
    }
    if (lane == 0) {
        Erow[NB] = 0;
        Erun[NB] = 0;
    }
    __syncwarp();
    uint32_t anchor = 0, o = 0;
    if (S >= LZ4_MFLIMIT + 1 && S >= LZ4_LASTLITERALS + LZ4_L0_MINMATCH) {
        const uint32_t wlim = (S - LZ4_LASTLITERALS - LZ4_L0_MINMATCH) / 4;  // last probe word
        const uint32_t matchlimit = S - LZ4_LASTLITERALS;                    // match end bound
        uint32_t pos = 0;
        for (uint32_t guard = 0; guard <= NW; guard++) {
            const uint32_t w0 = (pos + 3) / 4;
            if (w0 > wlim) break;
            // first candidate word in [w0, wlim]
            uint32_t w = ~0u, isrow = 0;
            for (uint32_t qb = w0 >> 5; qb <= (wlim >> 5); qb += 32) {
                const uint32_t q = qb + lane;
                uint32_t crow = 0, crun = 0;
                if (q <= (wlim >> 5)) {
                    const uint32_t r0 = Erow[q], r1 = Erow[q + 1], u0 = Erun[q], u1 = Erun[q + 1];
                    // bits w .. w + LZ4_L0_MINWORDS - 1 all set
                    crow = r0;
                    crun = u0;
#pragma unroll
                    for (uint32_t k = 1; k < LZ4_L0_MINWORDS; k++) {
                        crow &= (r0 >> k) | (r1 << (32 - k));
                        crun &= (u0 >> k) | (u1 << (32 - k));
                    }
                    uint32_t keep = ~0u;
                    if (q == (w0 >> 5)) keep &= ~0u << (w0 & 31u);
                    if (q == (wlim >> 5)) keep &= (wlim & 31u) == 31u ? ~0u : ((2u << (wlim & 31u)) - 1u);
                    crow &= keep;
                    crun &= keep;
                }
                const uint32_t m = __ballot_sync(FULL, (crow | crun) != 0);
                if (m) {
                    const uint32_t fl = __ffs(m) - 1;
                    const uint32_t cr = __shfl_sync(FULL, crow, fl);
                    const uint32_t cu = __shfl_sync(FULL, crun, fl);
                    const uint32_t bit = __ffs(cr | cu) - 1;
                    w = (qb + fl) * 32 + bit;
                    isrow = (cr >> bit) & 1u;  // the previous bit-row wins a tie
                    break;
                }
            }
            if (w == ~0u) break;
            const uint32_t off = isrow ? rowlen : 4u;
            const uint32_t p0 = 4 * w;
            // whole words that still agree, then the agreeing bytes of the next
            const uint32_t cap = matchlimit / 4;
            const uint32_t wz =
                bitmap_first_zero(isrow ? Erow : Erun, w + LZ4_L0_MINWORDS, cap, lane);
            uint32_t len = 4 * (wz - w);
            if (4 * wz < matchlimit) {
                const uint32_t x = s32[wz] ^ s32[wz - off / 4];
                uint32_t eq = x ? ((uint32_t)(__ffs(x) - 1) >> 3) : 4u;
                if (eq > matchlimit - 4 * wz) eq = matchlimit - 4 * wz;
                len += eq;
            }
            uint32_t mp = p0;
            // back up over up to 3 equal bytes (never before the literal anchor)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (mp > anchor && mp > off && src[mp - 1] == src[mp - 1 - off]) {
                    mp--;
                    len++;
                }
            }
            o = lz4_emit(dst, o, src, anchor, mp, off, len, lane);
            anchor = mp + len;
            pos = anchor;
        }
    }
    o = lz4_emit_last(dst, o, src, anchor, S, lane);
    __syncwarp();
    return o;
}

// The level-0 parse as a graph.  A match of kind k (the previous bit-row, or
// a run of equal words) that starts anywhere in a maximal run of kind-k
// candidate words ends at the same place: three words after the run's last
// candidate (its equal words end there), capped at the match limit, plus the
// equal low bytes of the next word.  So the greedy parse only ever stands at
// such run ends (and at the block start).  Those are the nodes; a node's
// successor (the first candidate at or after its position, the kind the parse
// takes there and the candidate run holding it) does not depend on how the
// parse got there, so the warp computes every node's successor at once and
// the serial part of the parse is one shared load per sequence.  A block with
// LZ4_NODE_CAP nodes or more walks from candidate to match end instead; both
// give the same greedy parse, byte for byte.
constexpr uint32_t LZ4_NODE_CAP = 128;

// Shared scratch of lz4_encode_bitmap_fast: four 64-word bitmaps (candidates
// of either kind, bit-row candidates, and the last candidates of bit-row and
// of run candidate runs), the next-non-zero table of the first (65 entries in
// 80 bytes), two 64-entry rank tables and the node table.
constexpr uint32_t LZ4_FAST_SCRATCH = 4u * 64u * 4u + 80u + 2u * 64u + 4u * LZ4_NODE_CAP;

// First set bit in [from, to] of a 64-word shared bitmap, through its table
// nnz[k] = first k' >= k with bm[k'] != 0 (64 when none): one or two
// broadcast loads instead of a warp vote.  ~0u when none.
BSG_D uint32_t smap_first_set(const uint32_t *bm, const uint8_t *nnz, uint32_t from, uint32_t to)
{
    if (from > to) return ~0u;
    uint32_t k = from >> 5;
    uint32_t m = bm[k] & (~0u << (from & 31u));
    if (m == 0) {
        k = nnz[k + 1];
        if (k >= 64) return ~0u;
        m = bm[k];
    }
    const uint32_t w = 32u * k + (uint32_t)(__ffs(m) - 1);
    return w <= to ? w : ~0u;
}

// A lane's two words (k = lane, lane + 32) of a 64-word bitmap into shared
// memory with its next-non-zero table.
BSG_D void smap_store(uint32_t *bm, uint8_t *nnz, const uint32_t (&w)[2], uint32_t lane)
{
    bm[lane] = w[0];
    bm[lane + 32] = w[1];
    const uint32_t b0 = __ballot_sync(FULL, w[0] != 0), b1 = __ballot_sync(FULL, w[1] != 0);
#pragma unroll
    for (uint32_t j = 0; j < 2; j++) {
        const uint32_t k = lane + 32u * j;
        // set words at or after k: bits k.. of the 64-bit mask b1:b0
        const uint32_t lo = j == 0 ? (b0 >> lane) : 0u;
        const uint32_t hi = j == 0 ? b1 : (b1 >> lane);
        uint32_t nk;
        if (j == 0)
            nk = lo ? k + (uint32_t)(__ffs(lo) - 1) : (hi ? 32u + (uint32_t)(__ffs(hi) - 1) : 64u);
        else
            nk = hi ? k + (uint32_t)(__ffs(hi) - 1) : 64u;
        nnz[k] = (uint8_t)nk;
    }
    if (lane == 0) nnz[64] = 64;
}

// Bit w of the result: bit w of c set and bit w + 1 clear (the last of a run
// of set bits), for a lane's two words of a 64-word bitmap (word lane + 32 j
// in c[j]); bits past word 63 count as clear.
BSG_D void run_ends(const uint32_t (&c)[2], uint32_t (&e)[2], uint32_t lane)
{
    const uint32_t n0 = __shfl_down_sync(FULL, c[0], 1), n1 = __shfl_down_sync(FULL, c[1], 1);
    const uint32_t w32 = __shfl_sync(FULL, c[1], 0);
    const uint32_t h0 = lane == 31 ? w32 : n0, h1 = lane == 31 ? 0u : n1;
    e[0] = c[0] & ~((c[0] >> 1) | (h0 << 31));
    e[1] = c[1] & ~((c[1] >> 1) | (h1 << 31));
}

// Equality bitmaps of a block of NW = 32 NB words (NB <= 64) in shared
// memory: bit w of Erow set when word w equals word w - R (the bit-row
// above; none for R = 0), of Erun when it equals word w - 1; bitmap word k
// kept by lane k mod 32 in [k / 32].
BSG_D void lz4_eq_bitmaps(const uint32_t *s32, uint32_t NB, uint32_t R, uint32_t lane,
                          uint32_t (&Erow)[2], uint32_t (&Erun)[2])
{
    // Both neighbours are read from shared memory; words without one (w < R,
    // w = 0) read some word of the block instead and have their bits cleared
    // after the loop.
    Erow[0] = Erow[1] = Erun[0] = Erun[1] = 0u;
#pragma unroll
    for (uint32_t j = 0; j < 2; j++) {
        const uint32_t kend = NB < 32 * (j + 1) ? (NB > 32 * j ? NB - 32 * j : 0u) : 32u;
#pragma unroll 4
        for (uint32_t kk = 0; kk < kend; kk++) {
            const uint32_t w = 32 * (32 * j + kk) + lane;
            const uint32_t x = s32[w];
            const uint32_t xp = s32[w > 0 ? w - 1 : 0u];
            const uint32_t xr = s32[w > R ? w - R : 0u];
            const uint32_t row = __ballot_sync(FULL, x == xr);
            const uint32_t run = __ballot_sync(FULL, x == xp);
            if (lane == kk) {
                Erow[j] = row;
                Erun[j] = run;
            }
        }
    }
    // no word before word 0, no bit-row before words 0 .. R - 1 (none at all for R = 0)
    if (lane == 0) Erun[0] &= ~1u;
#pragma unroll
    for (uint32_t j = 0; j < 2; j++) {
        const uint32_t k0 = 32 * (lane + 32 * j);  // first word of bitmap word lane + 32 j
        if (R == 0 || k0 + 32 <= R) Erow[j] = 0u;
        else if (k0 < R) Erow[j] &= ~0u << (R - k0);
    }
}

// Level-0 encoder for the fast path (S a multiple of 128, at most 8192): the
// same parse as lz4_encode_bitmap.  From the equality bitmaps (two words per
// lane, as lz4_eq_bitmaps leaves them) it derives candidate bitmaps, kept in
// shared memory `scr` (LZ4_FAST_SCRATCH bytes, 4-byte aligned) with the
// candidate-run ends and their ranks, from which the warp builds the parse graph (node table: the
// node's position in 13 bits, the first candidate after it in 11, the
// successor node in 8, 255 for none).  The sequences are emitted 32 at a time
// in parallel: the parse collects up to 32 (literal start, match start, match
// length, offset) descriptors, one per lane; a warp scan of their encoded
// lengths places them; each lane writes its own token, length and offset
// bytes; the literal runs are copied one after another by the whole warp.
// NODE_CAP below LZ4_NODE_CAP only serves tests of the candidate walk.
template <uint32_t NODE_CAP = LZ4_NODE_CAP>
BSG_D uint32_t lz4_encode_bitmap_fast_eq(const uint8_t *src, uint32_t S, uint32_t rowlen,
                                         uint8_t *dst, uint32_t *scr, const uint32_t (&Erow)[2],
                                         const uint32_t (&Erun)[2])
{
    static_assert(NODE_CAP >= 1 && NODE_CAP <= LZ4_NODE_CAP && LZ4_NODE_CAP < 255, "node table");
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    const uint32_t NW = S / 4;
    const uint32_t R = (rowlen & 3u) ? 0u : rowlen / 4;
    // candidate bitmaps: bits w .. w + LZ4_L0_MINWORDS - 1 all set (LZ4_L0_MINMATCH
    // equal bytes)
    uint32_t Crow[2], Crun[2];
#pragma unroll
    for (int j = 0; j < 2; j++) {
        uint32_t nr = __shfl_down_sync(FULL, Erow[j], 1), nu = __shfl_down_sync(FULL, Erun[j], 1);
        const uint32_t nr1 = __shfl_sync(FULL, j == 0 ? Erow[1] : 0u, 0);
        const uint32_t nu1 = __shfl_sync(FULL, j == 0 ? Erun[1] : 0u, 0);
        if (lane == 31) {
            nr = nr1;
            nu = nu1;
        }
        Crow[j] = Erow[j];
        Crun[j] = Erun[j];
#pragma unroll
        for (uint32_t k = 1; k < LZ4_L0_MINWORDS; k++) {
            Crow[j] &= (Erow[j] >> k) | (nr << (32 - k));
            Crun[j] &= (Erun[j] >> k) | (nu << (32 - k));
        }
    }
    const uint32_t Cany[2] = {Crow[0] | Crun[0], Crow[1] | Crun[1]};
    uint32_t CEr[2], CEu[2];
    run_ends(Crow, CEr, lane);
    run_ends(Crun, CEu, lane);
    uint32_t *sCany = scr, *sCrow = scr + 64, *sCEr = scr + 128, *sCEu = scr + 192;
    uint8_t *nCany = reinterpret_cast<uint8_t *>(scr + 256);
    uint8_t *preR = nCany + 80, *preU = preR + 64;
    uint32_t *node = scr + 256 + (80 + 128) / 4;
    smap_store(sCany, nCany, Cany, lane);
    sCrow[lane] = Crow[0];
    sCrow[lane + 32] = Crow[1];
    sCEr[lane] = CEr[0];
    sCEr[lane + 32] = CEr[1];
    sCEu[lane] = CEu[0];
    sCEu[lane + 32] = CEu[1];
    // run ends of each kind in the words before word k (bit-row in the low,
    // run in the high 16 bits): the rank of a candidate run among its kind
    const uint32_t c0 = (uint32_t)__popc(CEr[0]) | ((uint32_t)__popc(CEu[0]) << 16);
    const uint32_t c1 = (uint32_t)__popc(CEr[1]) | ((uint32_t)__popc(CEu[1]) << 16);
    uint32_t i0 = c0, i1 = c1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t0 = __shfl_up_sync(FULL, i0, d), t1 = __shfl_up_sync(FULL, i1, d);
        if (lane >= (uint32_t)d) {
            i0 += t0;
            i1 += t1;
        }
    }
    const uint32_t tot0 = __shfl_sync(FULL, i0, 31);
    const uint32_t tot = __shfl_sync(FULL, i1, 31) + tot0;
    const uint32_t x0 = i0 - c0, x1 = i1 - c1 + tot0;  // exclusive, words lane and lane + 32
    const uint32_t Nr = tot & 0xffffu, N = Nr + (tot >> 16);
    const bool graph = N < NODE_CAP;  // nodes 0 .. N - 1 and the start, N
    if (graph) {
        preR[lane] = (uint8_t)x0;
        preR[lane + 32] = (uint8_t)x1;
        preU[lane] = (uint8_t)(x0 >> 16);
        preU[lane + 32] = (uint8_t)(x1 >> 16);
        // node ids in position order within each kind: the last word of a
        // bit-row candidate run first, then those of run candidate runs
#pragma unroll
        for (uint32_t j = 0; j < 2; j++) {
            const uint32_t wb = 32u * (lane + 32u * j), x = j ? x1 : x0;
            uint32_t m = j ? CEr[1] : CEr[0], id = x & 0xffffu;
            for (; m; m &= m - 1) node[id++] = wb + (uint32_t)(__ffs(m) - 1);
            m = j ? CEu[1] : CEu[0];
            id = Nr + (x >> 16);
            for (; m; m &= m - 1) node[id++] = wb + (uint32_t)(__ffs(m) - 1);
        }
    }
    __syncwarp();

    uint32_t anchor = 0, o = 0;
    if (S >= LZ4_MFLIMIT + 1 && S >= LZ4_LASTLITERALS + LZ4_L0_MINMATCH) {
        const uint32_t wlim = (S - LZ4_LASTLITERALS - LZ4_L0_MINMATCH) / 4;
        const uint32_t matchlimit = S - LZ4_LASTLITERALS;
        const uint32_t cap = matchlimit / 4;
        if (graph) {
            // each node's position and successor (a lane reads and rewrites
            // only its own entries)
            for (uint32_t id = lane; id <= N; id += 32) {
                uint32_t p = 0;
                if (id < N) {
                    uint32_t e = node[id] + LZ4_L0_MINWORDS;
                    if (e > cap) e = cap;
                    p = 4 * e;
                    if (p < matchlimit) {
                        const uint32_t x = s32[e] ^ s32[e - (id < Nr ? R : 1u)];
                        uint32_t eq = x ? ((uint32_t)(__ffs(x) - 1) >> 3) : 4u;
                        if (eq > matchlimit - p) eq = matchlimit - p;
                        p += eq;
                    }
                }
                const uint32_t w = smap_first_set(sCany, nCany, (p + 3) / 4, wlim);
                uint32_t rec = p | (255u << 24);
                if (w != ~0u) {
                    // the previous bit-row wins a tie
                    const uint32_t wd = w >> 5, below = (1u << (w & 31u)) - 1u;
                    const bool row = (sCrow[wd] >> (w & 31u)) & 1u;
                    const uint32_t nx = row ? preR[wd] + (uint32_t)__popc(sCEr[wd] & below)
                                            : Nr + preU[wd] + (uint32_t)__popc(sCEu[wd] & below);
                    rec = p | (w << 13) | (nx << 24);
                }
                node[id] = rec;
            }
            __syncwarp();
        }
        static_assert(4 * LZ4_NODE_CAP <= 2 * 64 * 4, "jump tables in the run-end bitmaps");
        uint8_t *jmp = reinterpret_cast<uint8_t *>(sCEr);
        if (graph) {
            // jump tables: jmp[b * LZ4_NODE_CAP + x] = the node 2^(b + 1)
            // steps after node x (255: past the end), in the space of the
            // run-end bitmaps, which the graph parse no longer reads
            for (uint32_t x = lane; x <= N; x += 32) {
                const uint32_t y = node[x] >> 24;
                jmp[x] = (uint8_t)(y == 255u ? 255u : node[y] >> 24);
            }
            __syncwarp();
#pragma unroll
            for (uint32_t b = 1; b < 4; b++) {
                const uint8_t *jp = jmp + (b - 1) * LZ4_NODE_CAP;
                for (uint32_t x = lane; x <= N; x += 32) {
                    const uint32_t y = jp[x];
                    jmp[b * LZ4_NODE_CAP + x] = (uint8_t)(y == 255u ? 255u : jp[y]);
                }
                __syncwarp();
            }
        }
        uint32_t x0 = N;  // graph: the node the next 32 sequences start from
        uint32_t pos = 0;
        bool more = true;
        for (uint32_t guard = 0; more && guard <= NW; guard++) {
            // up to 32 sequences; lane k keeps the k-th
            uint32_t my_anchor = 0, my_mp = 0, my_len = 0, my_off = 0, n = 0;
            if (graph) {
                // lane k: the node k steps after x0 (the start of its
                // sequence) and the node after that (its end)
                uint32_t x = x0;
                if (lane & 1u) x = node[x] >> 24;
#pragma unroll
                for (uint32_t b = 0; b < 4; b++)
                    if (((lane >> (b + 1)) & 1u) && x != 255u) x = jmp[b * LZ4_NODE_CAP + x];
                const uint32_t rec = x != 255u ? node[x] : 0u;
                const uint32_t nx = x != 255u ? rec >> 24 : 255u;
                if (nx != 255u) {
                    const uint32_t nrec = node[nx];
                    my_anchor = rec & 8191u;
                    my_mp = 4 * ((rec >> 13) & 2047u);
                    my_len = (nrec & 8191u) - my_mp;
                    my_off = nx < Nr ? rowlen : 4u;
                }
                n = (uint32_t)__popc(__ballot_sync(FULL, nx != 255u));
                if (n) pos = __shfl_sync(FULL, my_mp + my_len, n - 1);
                x0 = __shfl_sync(FULL, nx, 31);
                more = n == 32 && x0 != 255u;
            } else {
                for (; n < 32; n++) {
                    uint32_t mp, len, off;
                    const uint32_t w = smap_first_set(sCany, nCany, (pos + 3) / 4, wlim);
                    if (w == ~0u) {
                        more = false;
                        break;
                    }
                    // the previous bit-row wins a tie
                    const bool row = (sCrow[w >> 5] >> (w & 31u)) & 1u;
                    const uint32_t *ce = row ? sCEr : sCEu;
                    // the candidate run holding w ends at or after it
                    uint32_t wd = w >> 5, m = ce[wd] & (~0u << (w & 31u));
                    while (m == 0 && wd < 63) m = ce[++wd];
                    uint32_t e = m ? 32 * wd + (uint32_t)(__ffs(m) - 1) + LZ4_L0_MINWORDS : cap;
                    if (e > cap) e = cap;
                    off = row ? rowlen : 4u;
                    mp = 4 * w;
                    len = 4 * (e - w);
                    if (4 * e < matchlimit) {
                        const uint32_t x = s32[e] ^ s32[e - off / 4];
                        uint32_t eq = x ? ((uint32_t)(__ffs(x) - 1) >> 3) : 4u;
                        if (eq > matchlimit - 4 * e) eq = matchlimit - 4 * e;
                        len += eq;
                    }
                    if (lane == n) {
                        my_anchor = pos;
                        my_mp = mp;
                        my_len = len;
                        my_off = off;
                    }
                    pos = mp + len;  // the backward extension below leaves the match end alone
                }
            }
            // each lane backs its match up over up to 3 equal bytes (never
            // before its literal anchor), off the parse's critical path
            if (lane < n && my_mp > my_anchor && my_mp > my_off) {
                const uint32_t x = ld32u(src, my_mp - 4) ^ ld32u(src, my_mp - 4 - my_off);
                uint32_t back = (x ? __clz(x) : 32u) >> 3;
                if (back > 3) back = 3;
                if (back > my_mp - my_anchor) back = my_mp - my_anchor;
                if (back > my_mp - my_off) back = my_mp - my_off;
                my_mp -= back;
                my_len += back;
            }
            // emit the n sequences of this batch
            const bool mine = lane < n;
            const uint32_t LL = mine ? my_mp - my_anchor : 0u;
            const uint32_t ML = mine ? my_len - LZ4_MINMATCH : 0u;
            const uint32_t nll = lz4_ext_count(LL), nml = lz4_ext_count(ML);
            const uint32_t total = mine ? 1 + nll + LL + 2 + nml : 0u;
            uint32_t incl = total;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(FULL, incl, d);
                if (lane >= (uint32_t)d) incl += t;
            }
            const uint32_t base = o + incl - total;
            if (mine) {
                dst[base] = (uint8_t)(((LL < 15 ? LL : 15) << 4) | (ML < 15 ? ML : 15));
                for (uint32_t k = 0; k < nll; k++)
                    dst[base + 1 + k] = k + 1 < nll ? 255u : (uint8_t)((LL - 15) % 255u);
                const uint32_t tr = base + 1 + nll + LL;
                dst[tr] = (uint8_t)(my_off & 255u);
                dst[tr + 1] = (uint8_t)(my_off >> 8);
                for (uint32_t k = 0; k < nml; k++)
                    dst[tr + 2 + k] = k + 1 < nml ? 255u : (uint8_t)((ML - 15) % 255u);
            }
            warp_copy_ranges(dst, src, n, my_anchor, base + 1 + nll, LL, lane);
            o += __shfl_sync(FULL, incl, 31);
            anchor = pos;
        }
    }
    __syncwarp();
    o = lz4_emit_last(dst, o, src, anchor, S, lane);
    __syncwarp();
    return o;
}

// The same, building its equality bitmaps from the block in shared memory.
template <uint32_t NODE_CAP = LZ4_NODE_CAP>
BSG_D uint32_t lz4_encode_bitmap_fast(const uint8_t *src, uint32_t S, uint32_t rowlen, uint8_t *dst,
                                      uint32_t *scr)
{
    uint32_t Erow[2], Erun[2];
    lz4_eq_bitmaps(reinterpret_cast<const uint32_t *>(src), S / 128, (rowlen & 3u) ? 0u : rowlen / 4,
                   threadIdx.x & 31u, Erow, Erun);
    return lz4_encode_bitmap_fast_eq<NODE_CAP>(src, S, rowlen, dst, scr, Erow, Erun);
}

// Warp-parallel read of 255-continued length bytes at src[ip..]; adds them to
// *len.  Returns false if the bytes run past index `clen` (the stream end).
BSG_D bool lz4_read_len(const uint8_t *src, uint32_t clen, uint32_t &ip, uint32_t &len,
                        uint32_t lane)
{
    // nearly always one byte below 255: no warp vote
    if (ip < clen) {
        const uint32_t b0 = src[ip];
        if (b0 != 255u) {
            len += b0;
            ip += 1;
            return true;
        }
    }
    for (uint32_t g = 0; g <= clen; g += 32) {
        uint32_t idx = ip + lane;
        uint32_t b = idx < clen ? src[idx] : 0u;
        uint32_t m = __ballot_sync(FULL, b != 255u);
        if (m == 0) {
            len += 255u * 32u;
            ip += 32;
            continue;
        }
        uint32_t f = __ffs(m) - 1;
        if (ip + f >= clen) return false;
        len += 255u * f + __shfl_sync(FULL, b, f);
        ip += f + 1;
        return true;
    }
    return false;
}

// Copy a match of ML bytes at distance off to dst[op..] (off <= op).  Reads
// of an overlapping match (off < ML) only see bytes written in earlier rounds.
BSG_D void lz4_match_copy(uint8_t *dst, uint32_t op, uint32_t off, uint32_t ML, uint32_t lane)
{
    if (off >= ML) {
        warp_copy(dst, op, dst, op - off, ML, lane);
    } else if (off == 1 || off == 2 || off == 4) {
        // period dividing 4: every aligned output word holds the same value
        warp_fill_pattern(dst, op, off, ML, lane);
    } else if (off >= 32) {
        // steps of at most `off` bytes never read what the same step writes
        const uint32_t W = off < 512u ? off : 512u;
        for (uint32_t base = 0; base < ML; base += W) {
            warp_copy(dst, op + base, dst, op + base - off, ML - base < W ? ML - base : W, lane);
            __syncwarp();
        }
    } else {
        // period off < 32: out[op + i] = out[op - off + i mod off]
        const uint32_t W = off * (32u / off);
        const uint8_t v = lane < W ? dst[op - off + lane % off] : 0;
        __syncwarp();
        for (uint32_t base = 0; base < ML; base += W) {
            const uint32_t k = base + lane;
            if (lane < W && k < ML) dst[op + k] = v;
        }
    }
}

// Strict decode of the clen bytes src[ip0 ..] into exactly S bytes of dst
// (src and dst word-aligned shared buffers; src readable 8 bytes past the
// end).  Returns 0, or a nonzero code for: input ending early (1), a literal
// run overrunning the output (2), a bad offset or match length, or a match
// breaking the end-of-block rules (3), a final length other than S (6).
// The token and the offset are each read together with the byte after them
// (one funnel-shifted word), so a length of 15..269 costs no extra read.
BSG_D int lz4_decode_warp(const uint8_t *src, uint32_t ip0, uint32_t clen, uint8_t *dst,
                          uint32_t S)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t end = ip0 + clen;
    uint32_t ip = ip0, op = 0;
    // every pass consumes at least its token byte, so the loop ends
    while (true) {
        if (ip >= end) return 1;
        const uint32_t t4 = ld32u(src, ip);
        const uint32_t token = t4 & 255u;
        uint32_t LL = token >> 4;
        ip += 1;
        if (LL == 15u) {
            const uint32_t b = (t4 >> 8) & 255u;
            if (b != 255u && ip < end) {
                LL += b;
                ip += 1;
            } else if (!lz4_read_len(src, end, ip, LL, lane)) {
                return 1;
            }
        }
        if (LL > end - ip) return 1;
        if (LL > S - op) return 2;
        warp_copy_ordered(dst, op, src, ip, LL, lane);
        ip += LL;
        op += LL;
        if (ip == end) break;
        if (end - ip < 2) return 1;
        const uint32_t o4 = ld32u(src, ip);
        const uint32_t off = o4 & 0xffffu;
        ip += 2;
        uint32_t ML = token & 15u;
        if (ML == 15u) {
            const uint32_t b = (o4 >> 16) & 255u;
            if (b != 255u && ip < end) {
                ML += b;
                ip += 1;
            } else if (!lz4_read_len(src, end, ip, ML, lane)) {
                return 1;
            }
        }
        ML += LZ4_MINMATCH;
        // (ML is below 2^31: at most 255 per stream byte)
        if ((off == 0) | (off > op) | (ML + LZ4_LASTLITERALS > S - op) | (op + LZ4_MFLIMIT > S))
            return 3;
        __syncwarp();
        lz4_match_copy(dst, op, off, ML, lane);
        op += ML;
        __syncwarp();
    }
    __syncwarp();
    return op == S ? 0 : 6;
}

#endif  // __CUDACC__ || BSG_WARP_EMU

}  // namespace bsg
