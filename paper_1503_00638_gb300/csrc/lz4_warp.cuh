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

#if defined(__CUDACC__) || defined(BSG_WARP_EMU)

// 4 bytes starting at byte q of a word-aligned shared buffer (little endian);
// reads the aligned words at q & ~3 and the next one
BSG_D uint32_t ld32u(const uint8_t *base, uint32_t q)
{
    const uint32_t *w = reinterpret_cast<const uint32_t *>(base);
    uint32_t i = q >> 2;
    return funnel_r(w[i], w[i + 1], (q & 3u) * 8u);
}

// Write one sequence (literals [anchor, mp), match of `len` bytes at
// distance `off`) at dst[o..]; returns the new output length.
BSG_D uint32_t lz4_emit(uint8_t *dst, uint32_t o, const uint8_t *src, uint32_t anchor,
                        uint32_t mp, uint32_t off, uint32_t len, uint32_t lane)
{
    uint32_t LL = mp - anchor;
    uint32_t ML = len - LZ4_MINMATCH;
    uint32_t nll = LL >= 15 ? (LL - 15) / 255 + 1 : 0;
    uint32_t nml = ML >= 15 ? (ML - 15) / 255 + 1 : 0;
    uint32_t hdr = 1 + nll;
    uint32_t total = hdr + LL + 2 + nml;
    uint32_t token = ((LL < 15 ? LL : 15) << 4) | (ML < 15 ? ML : 15);
    for (uint32_t idx = lane; idx < total; idx += 32) {
        uint32_t b;
        if (idx == 0) {
            b = token;
        } else if (idx < hdr) {
            b = (idx < hdr - 1) ? 255u : (LL - 15) % 255u;
        } else if (idx < hdr + LL) {
            b = src[anchor + idx - hdr];
        } else if (idx == hdr + LL) {
            b = off & 255u;
        } else if (idx == hdr + LL + 1) {
            b = off >> 8;
        } else {
            uint32_t j = idx - hdr - LL - 2;
            b = (j < nml - 1) ? 255u : (ML - 15) % 255u;
        }
        dst[o + idx] = (uint8_t)b;
    }
    return o + total;
}

// Literals-only last sequence [anchor, S).
BSG_D uint32_t lz4_emit_last(uint8_t *dst, uint32_t o, const uint8_t *src, uint32_t anchor,
                             uint32_t S, uint32_t lane)
{
    uint32_t LL = S - anchor;
    uint32_t nll = LL >= 15 ? (LL - 15) / 255 + 1 : 0;
    uint32_t hdr = 1 + nll;
    uint32_t total = hdr + LL;
    uint32_t token = (LL < 15 ? LL : 15) << 4;
    for (uint32_t idx = lane; idx < total; idx += 32) {
        uint32_t b;
        if (idx == 0)
            b = token;
        else if (idx < hdr)
            b = (idx < hdr - 1) ? 255u : (LL - 15) % 255u;
        else
            b = src[anchor + idx - hdr];
        dst[o + idx] = (uint8_t)b;
    }
    return o + total;
}

// Encode src[0, S) (word aligned, readable up to S + 8) into dst (capacity
// lz4_bound(S)).  Probes 32 word-aligned positions per step with a table of
// the last aligned position of each 4-byte hash (cleared here) plus the
// nearest earlier lane holding the same word; takes the first verified
// match, extends it back by up to 3 bytes and forward warp-wide.  The result
// depends only on the bytes of the block.  Returns the compressed size, or
// 0xffffffff if the progress guard tripped (cannot happen for valid sizes).
template <int HBITS>
BSG_D uint32_t lz4_encode_warp(const uint8_t *src, uint32_t S, uint8_t *dst, uint32_t *table)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lt = lanemask_lt();
    for (uint32_t i = lane; i < (1u << HBITS); i += 32) table[i] = 0;
    __syncwarp();
    uint32_t anchor = 0, o = 0;
    if (S >= LZ4_MFLIMIT + 1) {
        const uint32_t mflimit = S - LZ4_MFLIMIT;       // last allowed match start
        const uint32_t matchlimit = S - LZ4_LASTLITERALS;  // match end bound
        uint32_t pos = 0, fails = 0;
        const uint32_t guard = S / 4 + 8;
        uint32_t it = 0;
        while (pos <= mflimit) {
            if (++it > guard) return 0xffffffffu;
            uint32_t sh = fails / LZ4_ACCEL_WINDOWS;
            uint32_t step = 4u << (sh < 2 ? sh : 2);
            uint32_t p = pos + step * lane;
            bool valid = p <= mflimit;
            uint32_t w = valid ? *reinterpret_cast<const uint32_t *>(src + p) : 0u;
            uint32_t h = (w * 2654435761u) >> (32 - HBITS);
            int32_t cand = valid ? (int32_t)table[h] - 1 : -1;
            uint32_t vmask = __ballot_sync(FULL, valid);
            uint32_t same = __match_any_sync(FULL, w) & vmask & lt;
            bool intra = valid && same != 0;
            if (intra) cand = (int32_t)(pos + step * (31 - __clz(same)));
            bool ok = valid && cand >= 0 &&
                      (intra || *reinterpret_cast<const uint32_t *>(src + cand) == w);
            uint32_t mm = __ballot_sync(FULL, ok);
            if (mm == 0) {
                if (valid) atomicMax(&table[h], p + 1);
                __syncwarp();
                fails++;
                pos += step * 32;
                continue;
            }
            uint32_t fl = __ffs(mm) - 1;
            if (valid && lane <= fl) atomicMax(&table[h], p + 1);
            uint32_t p0 = pos + step * fl;
            uint32_t mp = p0;
            uint32_t mc = (uint32_t)__shfl_sync(FULL, cand, fl);
            // back up over up to 3 equal bytes (never before the literal anchor)
#pragma unroll
            for (int b = 0; b < 3; b++) {
                if (mp > anchor && mc > 0 && src[mp - 1] == src[mc - 1]) {
                    mp--;
                    mc--;
                }
            }
            uint32_t len = p0 + 4 - mp;
            // extend forward, 128 bytes per step
            for (uint32_t g2 = 0; g2 < S; g2 += 128) {
                uint32_t q = mp + len + 4 * lane;
                int room = (int)matchlimit - (int)q;
                uint32_t eq = 0;
                if (room > 0) {
                    uint32_t x = ld32u(src, q) ^ ld32u(src, mc + len + 4 * lane);
                    eq = x ? ((uint32_t)(__ffs(x) - 1) >> 3) : 4u;
                    if ((int)eq > room) eq = (uint32_t)room;
                }
                uint32_t stop = __ballot_sync(FULL, eq < 4);
                if (stop == 0) {
                    len += 128;
                    continue;
                }
                uint32_t sl = __ffs(stop) - 1;
                len += 4 * sl + __shfl_sync(FULL, eq, sl);
                break;
            }
            __syncwarp();
            o = lz4_emit(dst, o, src, anchor, mp, mp - mc, len, lane);
            anchor = mp + len;
            pos = (anchor + 3u) & ~3u;
            fails = 0;
        }
    }
    o = lz4_emit_last(dst, o, src, anchor, S, lane);
    __syncwarp();
    return o;
}

// Warp-parallel read of 255-continued length bytes at src[ip..]; adds them to
// *len.  Returns false if the bytes run past clen.
BSG_D bool lz4_read_len(const uint8_t *src, uint32_t clen, uint32_t &ip, uint32_t &len,
                        uint32_t lane)
{
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

// Strict decode of src[0, clen) into exactly S bytes of dst.  Returns 0, or
// a nonzero code for: input ending early, a literal run or match overrunning
// the output, offset 0 or before the block start, a match breaking the
// end-of-block rules, or a final length other than S.
BSG_D int lz4_decode_warp(const uint8_t *src, uint32_t clen, uint8_t *dst, uint32_t S)
{
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t ip = 0, op = 0;
    for (uint32_t guard = 0; guard <= clen; guard++) {
        if (ip >= clen) return 1;
        uint32_t token = src[ip++];
        uint32_t LL = token >> 4;
        if (LL == 15 && !lz4_read_len(src, clen, ip, LL, lane)) return 1;
        if (LL > clen - ip) return 1;
        if (LL > S - op) return 2;
        for (uint32_t k = lane; k < LL; k += 32) dst[op + k] = src[ip + k];
        ip += LL;
        op += LL;
        if (ip == clen) break;
        if (clen - ip < 2) return 1;
        uint32_t off = (uint32_t)src[ip] | ((uint32_t)src[ip + 1] << 8);
        ip += 2;
        if (off == 0) return 3;
        if (off > op) return 4;
        uint32_t ML = token & 15u;
        if (ML == 15 && !lz4_read_len(src, clen, ip, ML, lane)) return 1;
        ML += LZ4_MINMATCH;
        if (ML > S - op) return 5;
        if (op + LZ4_MFLIMIT > S || op + ML + LZ4_LASTLITERALS > S) return 7;
        __syncwarp();
        if (off >= 32) {
            for (uint32_t base = 0; base < ML; base += 32) {
                uint32_t k = base + lane;
                if (k < ML) dst[op + k] = dst[op + k - off];
                __syncwarp();
            }
        } else {
            uint32_t W = off * (32u / off);
            uint8_t v = lane < W ? dst[op - off + lane % off] : 0;
            __syncwarp();
            for (uint32_t base = 0; base < ML; base += W) {
                uint32_t k = base + lane;
                if (lane < W && k < ML) dst[op + k] = v;
            }
        }
        op += ML;
        __syncwarp();
    }
    __syncwarp();
    return op == S ? 0 : 6;
}

#endif  // __CUDACC__ || BSG_WARP_EMU

}  // namespace bsg
