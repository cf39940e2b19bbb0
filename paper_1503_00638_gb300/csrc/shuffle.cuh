// Bitshuffle transposes of one block in shared memory (Sec. 4.2, Sec. 6
// step 4).  Element e's bit r (r = 8 * byte + bit, little-endian, LSB first
// as in the caption of Fig. f:bits) goes to bit-row r: byte r * (B/8) + e/8,
// bit e % 8.
//
// Fast paths (es = 4 and es = 8, B a multiple of 32): each lane takes a group
// of 32 consecutive elements, reads them from shared memory in 16-byte chunks
// in a lane-rotated order (conflict-free banks), transposes 32 x 32 bits in
// registers and undoes the rotation with one funnel shift per output word.
// es = 2 (B a multiple of 64) pairs words by byte permutes into the same
// 32 x 32 transpose; es = 1 (B a multiple of 32) transposes 8 x 8 bit
// matrices in 64-bit words.  Other shapes take the byte-by-byte generic path.
#pragma once

#include "common.cuh"

namespace bsg {

BSG_HD bool shuffle_fast_ok(uint32_t es, uint32_t Bb)
{
    return (es == 4 || es == 8) && (Bb % 32u) == 0;
}

// src: Bb elements of 4 bytes (16-byte aligned); dst: 32 bit-rows of Bb/8 bytes
BSG_HD void shuffle4_fast(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 32;  // groups of 32 elements; also words per bit-row
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t g = lane; g < G; g += 32) {
        const uint8_t *grp = src + 128u * g;
        const uint32_t rot = g & 7u;
        uint32_t a[32];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            uint4 v = *reinterpret_cast<const uint4 *>(grp + 16u * ((k + rot) & 7u));
            a[4 * k] = v.x;
            a[4 * k + 1] = v.y;
            a[4 * k + 2] = v.z;
            a[4 * k + 3] = v.w;
        }
        // a[m] holds element (m + 4 rot) mod 32
        transpose32(a);
#pragma unroll
        for (int r = 0; r < 32; r++) d32[r * G + g] = rotl(a[r], 4u * rot);
    }
}

// src: 32 bit-rows of Bb/8 bytes; dst: Bb elements of 4 bytes
BSG_HD void unshuffle4_fast(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 32;
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    for (uint32_t g = lane; g < G; g += 32) {
        const uint32_t rot = g & 7u;
        uint32_t a[32];
#pragma unroll
        for (int r = 0; r < 32; r++) a[r] = rotr(s32[r * G + g], 4u * rot);
        // after the transpose a[m] holds element (m + 4 rot) mod 32
        transpose32(a);
        uint8_t *grp = dst + 128u * g;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            *reinterpret_cast<uint4 *>(grp + 16u * ((k + rot) & 7u)) =
                make_uint4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
        }
    }
}

// 8-byte elements: the low and high words of a group transpose separately
// into bit-rows 0..31 and 32..63.
BSG_HD void shuffle8_fast(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 32;
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t g = lane; g < G; g += 32) {
        const uint8_t *grp = src + 256u * g;
        const uint32_t rot = g & 15u;
        uint32_t lo[32], hi[32];
#pragma unroll
        for (int k = 0; k < 16; k++) {
            uint4 v = *reinterpret_cast<const uint4 *>(grp + 16u * ((k + rot) & 15u));
            lo[2 * k] = v.x;
            hi[2 * k] = v.y;
            lo[2 * k + 1] = v.z;
            hi[2 * k + 1] = v.w;
        }
        // lo[m], hi[m] hold element (m + 2 rot) mod 32
        transpose32(lo);
#pragma unroll
        for (int r = 0; r < 32; r++) d32[r * G + g] = rotl(lo[r], 2u * rot);
        transpose32(hi);
#pragma unroll
        for (int r = 0; r < 32; r++) d32[(32 + r) * G + g] = rotl(hi[r], 2u * rot);
    }
}

BSG_HD void unshuffle8_fast(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 32;
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    for (uint32_t g = lane; g < G; g += 32) {
        const uint32_t rot = g & 15u;
        uint32_t lo[32], hi[32];
#pragma unroll
        for (int r = 0; r < 32; r++) {
            lo[r] = rotr(s32[r * G + g], 2u * rot);
            hi[r] = rotr(s32[(32 + r) * G + g], 2u * rot);
        }
        transpose32(lo);
        transpose32(hi);
        uint8_t *grp = dst + 256u * g;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            *reinterpret_cast<uint4 *>(grp + 16u * ((k + rot) & 15u)) =
                make_uint4(lo[2 * k], hi[2 * k], lo[2 * k + 1], hi[2 * k + 1]);
        }
    }
}

// Generic paths: any es in {1,2,4,8} and Bb a multiple of 8.  One output byte
// per lane step, gathered from 8 input bytes.
BSG_HD void shuffle_generic(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t es,
                            uint32_t lane)
{
    const uint32_t rowb = Bb / 8;
    const uint32_t S = Bb * es;
    for (uint32_t o = lane; o < S; o += 32) {
        uint32_t r = o / rowb, col = o - r * rowb;
        uint32_t byte = r >> 3, bit = r & 7u;
        uint32_t v = 0;
#pragma unroll
        for (uint32_t e = 0; e < 8; e++)
            v |= ((uint32_t)(src[(8 * col + e) * es + byte] >> bit) & 1u) << e;
        dst[o] = (uint8_t)v;
    }
}

BSG_HD void unshuffle_generic(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t es,
                            uint32_t lane)
{
    const uint32_t rowb = Bb / 8;
    const uint32_t S = Bb * es;
    for (uint32_t o = lane; o < S; o += 32) {
        uint32_t e = o / es, byte = o - e * es;
        uint32_t v = 0;
#pragma unroll
        for (uint32_t bit = 0; bit < 8; bit++)
            v |= ((uint32_t)(src[(8 * byte + bit) * rowb + e / 8] >> (e & 7u)) & 1u) << bit;
        dst[o] = (uint8_t)v;
    }
}

#if defined(__CUDACC__) || defined(BSG_WARP_EMU)
// Un-transpose a block of 4-byte elements in place (buf holds 32 bit-rows of
// Bb/8 bytes; afterwards the Bb elements), for Bb <= 1024 (one group of 32
// elements per lane) or Bb == 2048 (two).  With 64 groups, group g's output
// is words [32 g, 32 g + 32) and row r of group g is word 64 r + g: the first
// groups' outputs (g < 32, the first half) overwrite only rows 0..15, so a
// lane reads rows 0..15 of both its groups and rows 16..31 of its first group
// (48 values) before anything is written, then the rest.
BSG_D void unshuffle4_inplace(uint8_t *buf, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 32;
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(buf);
    auto store_group = [&](uint32_t g, uint32_t (&a)[32]) {
        transpose32(a);  // a[m] holds element (m + 4 rot) mod 32
        const uint32_t rot = g & 7u;
        uint8_t *grp = buf + 128u * g;
#pragma unroll
        for (int k = 0; k < 8; k++)
            *reinterpret_cast<uint4 *>(grp + 16u * ((k + rot) & 7u)) =
                make_uint4(a[4 * k], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
    };
    const uint32_t g0 = lane, s0 = 4u * (g0 & 7u);
    uint32_t a[32];
    if (G <= 32) {
        if (g0 < G) {
#pragma unroll
            for (int r = 0; r < 32; r++) a[r] = rotr(s32[r * G + g0], s0);
        }
        __syncwarp();
        if (g0 < G) store_group(g0, a);
        return;
    }
    // G == 64
    const uint32_t g1 = lane + 32u, s1 = 4u * (g1 & 7u);
    uint32_t b[32];
#pragma unroll
    for (int r = 0; r < 32; r++) a[r] = rotr(s32[r * 64 + g0], s0);
#pragma unroll
    for (int r = 0; r < 16; r++) b[r] = rotr(s32[r * 64 + g1], s1);
    __syncwarp();
    store_group(g0, a);
#pragma unroll
    for (int r = 16; r < 32; r++) b[r] = rotr(s32[r * 64 + g1], s1);
    __syncwarp();
    store_group(g1, b);
}

// Same for 8-byte elements and at most 32 groups (one per lane).
BSG_D void unshuffle8_inplace(uint8_t *buf, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 32;
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(buf);
    const uint32_t g = lane, rot = g & 15u;
    uint32_t lo[32], hi[32];
    if (g < G) {
#pragma unroll
        for (int r = 0; r < 32; r++) {
            lo[r] = rotr(s32[r * G + g], 2u * rot);
            hi[r] = rotr(s32[(32 + r) * G + g], 2u * rot);
        }
    }
    __syncwarp();
    if (g < G) {
        transpose32(lo);
        transpose32(hi);
        uint8_t *grp = buf + 256u * g;
#pragma unroll
        for (int k = 0; k < 16; k++)
            *reinterpret_cast<uint4 *>(grp + 16u * ((k + rot) & 15u)) =
                make_uint4(lo[2 * k], hi[2 * k], lo[2 * k + 1], hi[2 * k + 1]);
    }
}

// Bit-transpose a block of 4-byte elements in place (buf holds Bb elements;
// afterwards its 32 bit-rows of Bb/8 bytes), for Bb <= 1024 (one group of 32
// elements per lane) or Bb == 2048 (two).  Each group's 32 values pass through
// `fix(g, a)` before the transpose (the hook that rounds visibility data);
// a[m] then holds element (m + 4 (g & 7)) mod 32 of group g.
//
// With 64 groups, row r of group g is word 64 r + g: rows 0..15 of the first
// groups (g < 32) fall in the first half of the buffer, which holds only the
// first groups' inputs, so they are written before the second groups are
// read, and at most 48 values per lane are live.
template <class Fix>
BSG_D void shuffle4_inplace(uint8_t *buf, uint32_t Bb, uint32_t lane, Fix fix)
{
    const uint32_t G = Bb / 32;
    uint32_t *d32 = reinterpret_cast<uint32_t *>(buf);
    auto read_group = [&](uint32_t g, uint32_t (&a)[32]) {
        const uint8_t *grp = buf + 128u * g;
        const uint32_t rot = g & 7u;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            uint4 v = *reinterpret_cast<const uint4 *>(grp + 16u * ((k + rot) & 7u));
            a[4 * k] = v.x;
            a[4 * k + 1] = v.y;
            a[4 * k + 2] = v.z;
            a[4 * k + 3] = v.w;
        }
        fix(g, a);
        transpose32(a);
    };
    const uint32_t g0 = lane, rot0 = 4u * (g0 & 7u);
    uint32_t a[32];
    if (g0 < G) read_group(g0, a);
    __syncwarp();
    if (G <= 32) {
        if (g0 < G) {
#pragma unroll
            for (int r = 0; r < 32; r++) d32[r * G + g0] = rotl(a[r], rot0);
        }
        return;
    }
    // G == 64
#pragma unroll
    for (int r = 0; r < 16; r++) d32[r * 64 + g0] = rotl(a[r], rot0);
    const uint32_t g1 = lane + 32u, rot1 = 4u * (g1 & 7u);
    uint32_t b[32];
    read_group(g1, b);
    __syncwarp();
#pragma unroll
    for (int r = 16; r < 32; r++) d32[r * 64 + g0] = rotl(a[r], rot0);
#pragma unroll
    for (int r = 0; r < 32; r++) d32[r * 64 + g1] = rotl(b[r], rot1);
}

// shuffle4_inplace for Bb == 2048 that also returns the level-0 LZ4
// encoder's equality bitmaps of the bit-rows it writes, as
// lz4_eq_bitmaps computes them from shared memory: bit w of Erow set when
// word w of the rows equals word w - 64 (the same group one bit-row up),
// of Erun when it equals word w - 1; bitmap word k (words 32 k .. 32 k + 31)
// kept by lane k mod 32 in [k / 32].  Word 64 r + 32 j + lane is row r of
// group 32 j + lane, so each stored word is compared as it is stored with
// the lane's previous row (same lane) and with the lane before (a shuffle);
// the first word of each half-row, whose left neighbour is the other half's
// last group, is compared from shared memory after the stores.
template <class Fix>
BSG_D void shuffle4_inplace_eq(uint8_t *buf, uint32_t lane, Fix fix, uint32_t (&Erow)[2],
                               uint32_t (&Erun)[2])
{
    uint32_t *d32 = reinterpret_cast<uint32_t *>(buf);
    auto read_group = [&](uint32_t g, uint32_t (&a)[32]) {
        const uint8_t *grp = buf + 128u * g;
        const uint32_t rot = g & 7u;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            uint4 v = *reinterpret_cast<const uint4 *>(grp + 16u * ((k + rot) & 7u));
            a[4 * k] = v.x;
            a[4 * k + 1] = v.y;
            a[4 * k + 2] = v.z;
            a[4 * k + 3] = v.w;
        }
        fix(g, a);
        transpose32(a);
    };
    const uint32_t rot = 4u * (lane & 7u);  // groups lane and lane + 32 share it
    Erow[0] = Erow[1] = Erun[0] = Erun[1] = 0u;
    auto put = [&](int r, uint32_t j, uint32_t v, uint32_t vup) {
        d32[r * 64 + 32 * j + lane] = v;
        const uint32_t left = __shfl_up_sync(FULL, v, 1);
        const uint32_t row = __ballot_sync(FULL, r > 0 && v == vup);
        const uint32_t run = __ballot_sync(FULL, v == left);  // lane 0: fixed below
        const uint32_t k = 2u * (uint32_t)r + j;
        if (lane == (k & 31u)) {
            Erow[k >> 5] = row;
            Erun[k >> 5] = run;
        }
    };
    uint32_t a[32];
    read_group(lane, a);
    __syncwarp();
    uint32_t up = 0;
#pragma unroll
    for (int r = 0; r < 16; r++) {
        const uint32_t v = rotl(a[r], rot);
        put(r, 0, v, up);
        up = v;
    }
    uint32_t b[32];
    read_group(lane + 32u, b);
    __syncwarp();
#pragma unroll
    for (int r = 16; r < 32; r++) {
        const uint32_t v = rotl(a[r], rot);
        put(r, 0, v, up);
        up = v;
    }
    up = 0;
#pragma unroll
    for (int r = 0; r < 32; r++) {
        const uint32_t v = rotl(b[r], rot);
        put(r, 1, v, up);
        up = v;
    }
    __syncwarp();
    // word 64 r + 32 j (r = lane) against word 64 r + 32 j - 1; none before word 0
    const uint32_t x0 = d32[64 * lane], p0 = lane ? d32[64 * lane - 1] : ~x0;
    const uint32_t x1 = d32[64 * lane + 32], p1 = d32[64 * lane + 31];
    const uint32_t f0 = __ballot_sync(FULL, x0 == p0), f1 = __ballot_sync(FULL, x1 == p1);
#pragma unroll
    for (uint32_t h = 0; h < 2; h++) {
        const uint32_t k = 32u * h + lane;  // bitmap word 2 r + j
        Erun[h] = (Erun[h] & ~1u) | ((((k & 1u) ? f1 : f0) >> (k >> 1)) & 1u);
    }
}

// 8-byte elements, at most 32 groups (one per lane).
BSG_D void shuffle8_inplace(uint8_t *buf, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 32;
    uint32_t *d32 = reinterpret_cast<uint32_t *>(buf);
    const uint32_t g = lane, rot = g & 15u;
    uint32_t lo[32], hi[32];
    if (g < G) {
        const uint8_t *grp = buf + 256u * g;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            uint4 v = *reinterpret_cast<const uint4 *>(grp + 16u * ((k + rot) & 15u));
            lo[2 * k] = v.x;
            hi[2 * k] = v.y;
            lo[2 * k + 1] = v.z;
            hi[2 * k + 1] = v.w;
        }
    }
    __syncwarp();
    if (g < G) {
        transpose32(lo);
        transpose32(hi);
#pragma unroll
        for (int r = 0; r < 32; r++) {
            d32[r * G + g] = rotl(lo[r], 2u * rot);
            d32[(32 + r) * G + g] = rotl(hi[r], 2u * rot);
        }
    }
}

// 2-byte elements: a lane takes a group of 64 elements (128 bytes, 32 words
// w_0..w_31, word w_j holding elements 2j and 2j + 1).  Pairing w_j with
// w_(j+16) by byte permutes gives 32 words P_n = e_n | e_(n+32) << 16, so one
// 32 x 32 transpose yields bit r of elements 0..31 in word r and of elements
// 32..63 in word 16 + r: the group's two words of bit-row r (16 rows of Bb/8
// bytes).  The 16-byte chunks are read in a lane-rotated order over all 8
// chunks (conflict-free banks): step k reads chunk c = (k + g) & 7 and its
// partner c ^ 4, so a pair arrives as (w_j, w_(j+16)) when c < 4 and swapped
// otherwise, and the byte-permute selectors follow (a per-lane choice).  The
// columns come out rotated by 8 (g & 3) bits, undone on the rows.
struct Shuf2Sel {
    uint32_t lo, hi;  // selectors giving the pair's low and high halves
};

BSG_HD Shuf2Sel shuf2_sel(uint32_t c)
{
    return c < 4 ? Shuf2Sel{0x5410u, 0x7632u} : Shuf2Sel{0x1054u, 0x3276u};
}

// Group g of 64 2-byte elements (128 bytes at grp, rot = g & 7) into a[],
// transposed: a[r] and a[16 + r] hold bit-row r of the group's first and
// second 32 elements, rotated left by 8 (g & 3) bits.
BSG_D void shuf2_read_group(const uint8_t *grp, uint32_t rot, uint32_t (&a)[32])
{
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t c = (k + rot) & 7u;
        const uint4 v = *reinterpret_cast<const uint4 *>(grp + 16u * c);
        const uint4 w = *reinterpret_cast<const uint4 *>(grp + 16u * (c ^ 4u));
        const Shuf2Sel sel = shuf2_sel(c);
        const uint32_t x[4] = {v.x, v.y, v.z, v.w}, y[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            a[8 * k + 2 * i] = bperm(x[i], y[i], sel.lo);
            a[8 * k + 2 * i + 1] = bperm(x[i], y[i], sel.hi);
        }
    }
    // a[n] = P_((n + 8 rot) mod 32)
    transpose32(a);
}

// Bit-rows r0 .. r1-1 of group g into `out` (16 bit-rows of 2 G words).
BSG_D void shuf2_put_rows(uint8_t *out, uint32_t G, uint32_t g, const uint32_t (&a)[32], int r0,
                          int r1)
{
    const uint32_t s = 8u * (g & 3u);
#pragma unroll
    for (int r = r0; r < r1; r++)
        *reinterpret_cast<uint2 *>(out + 4u * (2u * G * r + 2u * g)) =
            make_uint2(rotl(a[r], s), rotl(a[16 + r], s));
}

// Bb <= 2048 (G <= 32 groups of 64, one per lane) or Bb == 4096 (G == 64:
// rows 0..7 of the first 32 groups fall in the first half of the buffer and
// are written before the second groups are read; at most 48 live values).
BSG_D void shuffle2_inplace(uint8_t *buf, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 64;
    const uint32_t g0 = lane;
    uint32_t a[32];
    if (g0 < G) shuf2_read_group(buf + 128u * g0, g0 & 7u, a);
    __syncwarp();
    if (G <= 32) {
        if (g0 < G) shuf2_put_rows(buf, G, g0, a, 0, 16);
        return;
    }
    // G == 64
    shuf2_put_rows(buf, G, g0, a, 0, 8);
    const uint32_t g1 = lane + 32u;
    uint32_t b[32];
    shuf2_read_group(buf + 128u * g1, g1 & 7u, b);
    __syncwarp();
    shuf2_put_rows(buf, G, g0, a, 8, 16);
    shuf2_put_rows(buf, G, g1, b, 0, 16);
}

// From src to dst (Bb a multiple of 64, any number of groups).
BSG_D void shuffle2_fast(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 64;
    for (uint32_t g = lane; g < G; g += 32) {
        uint32_t a[32];
        shuf2_read_group(src + 128u * g, g & 7u, a);
        shuf2_put_rows(dst, G, g, a, 0, 16);
    }
}

// Bit-rows r0 .. r1-1 of group g from `in` (16 bit-rows of 2 G words).
BSG_D void unshuf2_get_rows(const uint8_t *in, uint32_t G, uint32_t g, uint32_t (&a)[32], int r0,
                            int r1)
{
    const uint32_t s = 8u * (g & 3u);
#pragma unroll
    for (int r = r0; r < r1; r++) {
        const uint2 v = *reinterpret_cast<const uint2 *>(in + 4u * (2u * G * r + 2u * g));
        a[r] = rotr(v.x, s);
        a[16 + r] = rotr(v.y, s);
    }
}

// The group's 64 elements from its 16 bit-rows in a[] to grp (rot = g & 7).
BSG_D void unshuf2_store_group(uint8_t *grp, uint32_t rot, uint32_t (&a)[32])
{
    transpose32(a);  // a[n] = P_((n + 8 rot) mod 32)
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t c = (k + rot) & 7u;
        // P_2j = lo(w_j) | lo(w_(j+16)) << 16, P_2j+1 = hi(w_j) | hi(w_(j+16)) << 16
        uint32_t x[4], y[4];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const uint32_t wj = bperm(a[8 * k + 2 * i], a[8 * k + 2 * i + 1], 0x5410u);
            const uint32_t wj16 = bperm(a[8 * k + 2 * i], a[8 * k + 2 * i + 1], 0x7632u);
            x[i] = c < 4 ? wj : wj16;
            y[i] = c < 4 ? wj16 : wj;
        }
        *reinterpret_cast<uint4 *>(grp + 16u * c) = make_uint4(x[0], x[1], x[2], x[3]);
        *reinterpret_cast<uint4 *>(grp + 16u * (c ^ 4u)) = make_uint4(y[0], y[1], y[2], y[3]);
    }
}

// Inverse of shuffle2_inplace (same shapes).  With G == 64 a lane reads all
// of its first group and rows 0..7 of its second (48 values) before anything
// is written.
BSG_D void unshuffle2_inplace(uint8_t *buf, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 64;
    const uint32_t g0 = lane;
    uint32_t a[32];
    if (G <= 32) {
        if (g0 < G) unshuf2_get_rows(buf, G, g0, a, 0, 16);
        __syncwarp();
        if (g0 < G) unshuf2_store_group(buf + 128u * g0, g0 & 7u, a);
        return;
    }
    // G == 64
    const uint32_t g1 = lane + 32u;
    uint32_t b[32];
    unshuf2_get_rows(buf, G, g0, a, 0, 16);
    unshuf2_get_rows(buf, G, g1, b, 0, 8);
    __syncwarp();
    unshuf2_store_group(buf + 128u * g0, g0 & 7u, a);
    unshuf2_get_rows(buf, G, g1, b, 8, 16);
    __syncwarp();
    unshuf2_store_group(buf + 128u * g1, g1 & 7u, b);
}

// From src to dst (Bb a multiple of 64, any number of groups).
BSG_D void unshuffle2_fast(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t lane)
{
    const uint32_t G = Bb / 64;
    for (uint32_t g = lane; g < G; g += 32) {
        uint32_t a[32];
        unshuf2_get_rows(src, G, g, a, 0, 16);
        unshuf2_store_group(dst + 128u * g, g & 7u, a);
    }
}

// 1-byte elements: 8 consecutive bytes form an 8 x 8 bit matrix (byte i =
// element i, bit j = bit-row j); its transpose (three delta swaps, the
// classic method for an 8 x 8 bit transpose in a 64-bit word) has in byte j
// the output byte of bit-row j for those 8 elements.  A lane takes 32
// elements (four such matrices, read as two 16-byte chunks in a
// lane-alternated order) and writes one word to each of the 8 bit-rows.
BSG_D uint64_t transpose8x8(uint64_t x)
{
    uint64_t t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
    x ^= t ^ (t << 7);
    t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
    x ^= t ^ (t << 14);
    t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
    x ^= t ^ (t << 28);
    return x;
}

// src: Bb bytes (16-byte aligned), dst: 8 bit-rows of Bb/8 bytes; Bb % 32 == 0
BSG_D void shuffle1_fast(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t lane)
{
    const uint32_t Q = Bb / 32;  // groups of 32 elements; also words per bit-row
    uint32_t *d32 = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t q = lane; q < Q; q += 32) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src + 32u * q);
        const uint32_t o = q & 1u;
        const uint4 u = s4[o], v = s4[o ^ 1u];
        const uint4 c0 = o ? v : u, c1 = o ? u : v;
        const uint64_t m[4] = {transpose8x8(((uint64_t)c0.y << 32) | c0.x),
                               transpose8x8(((uint64_t)c0.w << 32) | c0.z),
                               transpose8x8(((uint64_t)c1.y << 32) | c1.x),
                               transpose8x8(((uint64_t)c1.w << 32) | c1.z)};
#pragma unroll
        for (uint32_t r = 0; r < 8; r++) {
            uint32_t w = 0;
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) w |= (uint32_t)((m[k] >> (8 * r)) & 0xffu) << (8 * k);
            d32[r * Q + q] = w;
        }
    }
}

BSG_D void unshuffle1_fast(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t lane)
{
    const uint32_t Q = Bb / 32;
    const uint32_t *s32 = reinterpret_cast<const uint32_t *>(src);
    for (uint32_t q = lane; q < Q; q += 32) {
        uint64_t m[4] = {0, 0, 0, 0};
#pragma unroll
        for (uint32_t r = 0; r < 8; r++) {
            const uint32_t w = s32[r * Q + q];
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) m[k] |= (uint64_t)((w >> (8 * k)) & 0xffu) << (8 * r);
        }
#pragma unroll
        for (uint32_t k = 0; k < 4; k++) m[k] = transpose8x8(m[k]);
        const uint4 c0 = make_uint4((uint32_t)m[0], (uint32_t)(m[0] >> 32), (uint32_t)m[1],
                                    (uint32_t)(m[1] >> 32));
        const uint4 c1 = make_uint4((uint32_t)m[2], (uint32_t)(m[2] >> 32), (uint32_t)m[3],
                                    (uint32_t)(m[3] >> 32));
        uint4 *d4 = reinterpret_cast<uint4 *>(dst + 32u * q);
        if (q & 1u) {
            d4[1] = c1;
            d4[0] = c0;
        } else {
            d4[0] = c0;
            d4[1] = c1;
        }
    }
}

// One lane's share of a block transpose; a warp calls it with lanes 0..31.
BSG_D void shuffle_block(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t es,
                         uint32_t lane)
{
    if (es == 4 && Bb % 32u == 0)
        shuffle4_fast(src, dst, Bb, lane);
    else if (es == 8 && Bb % 32u == 0)
        shuffle8_fast(src, dst, Bb, lane);
    else if (es == 2 && Bb % 64u == 0)
        shuffle2_fast(src, dst, Bb, lane);
    else if (es == 1 && Bb % 32u == 0)
        shuffle1_fast(src, dst, Bb, lane);
    else
        shuffle_generic(src, dst, Bb, es, lane);
}

BSG_D void unshuffle_block(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t es,
                           uint32_t lane)
{
    if (es == 4 && Bb % 32u == 0)
        unshuffle4_fast(src, dst, Bb, lane);
    else if (es == 8 && Bb % 32u == 0)
        unshuffle8_fast(src, dst, Bb, lane);
    else if (es == 2 && Bb % 64u == 0)
        unshuffle2_fast(src, dst, Bb, lane);
    else if (es == 1 && Bb % 32u == 0)
        unshuffle1_fast(src, dst, Bb, lane);
    else
        unshuffle_generic(src, dst, Bb, es, lane);
}

// Whether a block can be bit-transposed in place by the register paths above.
BSG_HD bool shuffle_inplace_ok(uint32_t es, uint32_t Bb)
{
    if (es == 2) return Bb % 64u == 0 && (Bb <= 2048 || Bb == 4096);
    return Bb % 32u == 0 && ((es == 4 && (Bb <= 1024 || Bb == 2048)) || (es == 8 && Bb <= 1024));
}

// Whether a block can be un-transposed in place by the register paths above.
BSG_HD bool unshuffle_inplace_ok(uint32_t es, uint32_t Bb)
{
    return shuffle_inplace_ok(es, Bb);
}
#endif  // __CUDACC__ || BSG_WARP_EMU

}  // namespace bsg
