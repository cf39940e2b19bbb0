// Bitshuffle transposes of one block in shared memory (Sec. 4.2, Sec. 6
// step 4).  Element e's bit r (r = 8 * byte + bit, little-endian, LSB first
// as in the caption of Fig. f:bits) goes to bit-row r: byte r * (B/8) + e/8,
// bit e % 8.
//
// Fast paths (es = 4 and es = 8, B a multiple of 32): each lane takes a group
// of 32 consecutive elements, reads them from shared memory in 16-byte chunks
// in a lane-rotated order (conflict-free banks), transposes 32 x 32 bits in
// registers and undoes the rotation with one funnel shift per output word.
// Other element sizes and shapes take the byte-by-byte generic path.
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

// One lane's share of a block transpose; a warp calls it with lanes 0..31.
BSG_HD void shuffle_block(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t es,
                          uint32_t lane)
{
    if (es == 4 && Bb % 32u == 0)
        shuffle4_fast(src, dst, Bb, lane);
    else if (es == 8 && Bb % 32u == 0)
        shuffle8_fast(src, dst, Bb, lane);
    else
        shuffle_generic(src, dst, Bb, es, lane);
}

BSG_HD void unshuffle_block(const uint8_t *src, uint8_t *dst, uint32_t Bb, uint32_t es,
                            uint32_t lane)
{
    if (es == 4 && Bb % 32u == 0)
        unshuffle4_fast(src, dst, Bb, lane);
    else if (es == 8 && Bb % 32u == 0)
        unshuffle8_fast(src, dst, Bb, lane);
    else
        unshuffle_generic(src, dst, Bb, es, lane);
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

// Whether a block can be bit-transposed in place by the register paths above.
BSG_HD bool shuffle_inplace_ok(uint32_t es, uint32_t Bb)
{
    return Bb % 32u == 0 && ((es == 4 && (Bb <= 1024 || Bb == 2048)) || (es == 8 && Bb <= 1024));
}

// Whether a block can be un-transposed in place by the register paths above.
BSG_HD bool unshuffle_inplace_ok(uint32_t es, uint32_t Bb)
{
    return shuffle_inplace_ok(es, Bb);
}
#endif  // __CUDACC__ || BSG_WARP_EMU

}  // namespace bsg
