// The fast compress kernel (full blocks of at most 8 KiB, Sec. 4.2.1), shared
// by the translation units that instantiate it: kernels.cu for cubes and
// streams stored in order, tslow.cu for time-slowest cubes and for cubes
// whose time axis is not a multiple of 16.
#pragma once

#include "codec.cuh"

namespace bsg {

// One warp per CTA, persistent, one shared buffer: bulk-copy the block in
// (TS: gather it from a time-slowest cube), round + bit-transpose it in place
// through registers, LZ4-encode it into this warp's staging slot in global
// memory (it stays in L2), publish its size, and place the PREVIOUS block: by
// then its predecessors have long published theirs, so the look-back rarely
// waits.  GEN (4-byte elements of a cube only): int32 components, a
// compensated c or the full-covariance q table (see round_group and
// round_group_full).  PS (a cube whose time axis is not a multiple of 16, so
// 16-sample groups would straddle products): the samples are rounded one by
// one before the plain transpose, and with TS gathered one by one.
template <int LEVEL, int ES, bool GEN = false, bool TS = false, bool PS = false>
__global__ void __launch_bounds__(32, 20) compress_fast_kernel(const __grid_constant__ CodecArgs a)
{
    using L = FastPlan<LEVEL>;
    // a staged block comes back into the buffer and the encoder's scratch
    // after it (both free by then) for its placement
    static_assert(L::TMP + L::SCR >= r16(4 + lz4b(L::MAXB)), "placement buffer");
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
        // 2048 4-byte elements at level 0 (the CHIME-shaped default): the
        // transpose also yields the encoder's equality bitmaps
        const bool EQ = LEVEL == 0 && ES == 4 && !PS && Bb == 2048;
        uint32_t Erow[2], Erun[2];
        if (TS) {
            if (PS)
                gather_tslow_samples(a, tmp, tile, lane);
            else
                gather_tslow_block(a, tmp, tile, lane);
            __syncwarp();
        } else if (load_block(tmp, a.in + (uint64_t)tile * a.B * a.es, Bb * a.es, bar, lane)) {
            if (!mbar_wait_bounded(bar, parity) && lane == 0) set_status(a.status, BSGPU_ERR_TIMEOUT);
            parity ^= 1u;
        }
        if (ES == 2) {
            shuffle2_inplace(tmp, Bb, lane);
        } else if (ES == 8) {
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
        } else if (PS && a.vis.enabled) {
            // a time axis that is not a multiple of 16: the components are
            // rounded sample by sample in place, then transposed
            const uint32_t c0 = (uint32_t)(((uint64_t)tile * a.B) >> 1);
            if ((a.vis.T & 1u) == 0) {
                uint4 *b4 = reinterpret_cast<uint4 *>(tmp);
                reduce_run2(b4, b4, c0, Bb / 2, a.vis, lane);
            } else {
                uint2 *b2 = reinterpret_cast<uint2 *>(tmp);
                reduce_run(b2, b2, c0, Bb / 2, a.vis, lane);
            }
            __syncwarp();
            shuffle4_inplace(tmp, Bb, lane, NoRound{});
        } else if (a.vis.enabled) {
            const VisGroupRound<GEN> round{&a.vis, (uint32_t)(((uint64_t)tile * a.B) >> 1)};
            if (EQ)
                shuffle4_inplace_eq(tmp, lane, round, Erow, Erun);
            else
                shuffle4_inplace(tmp, Bb, lane, round);
        } else if (EQ) {
            shuffle4_inplace_eq(tmp, lane, NoRound{}, Erow, Erun);
        } else {
            shuffle4_inplace(tmp, Bb, lane, NoRound{});
        }
        __syncwarp();
        uint32_t cs;
        if (LEVEL == 0 && (Bb * ES) % 128u == 0) {
            if (!EQ)
                lz4_eq_bitmaps(reinterpret_cast<const uint32_t *>(tmp), Bb * ES / 128, Bb / 32, lane, Erow,
                               Erun);
            cs = lz4_encode_bitmap_fast_eq(tmp, Bb * ES, Bb / 8, slot0 + 4,
                                           static_cast<uint32_t *>(scratch), Erow, Erun);
            if (lane == 0) put_be32(slot0, cs);
            __syncwarp();
        } else {
            cs = compress_encode<LEVEL, L::HBITS>(a, Bb, tmp, slot0, scratch, lane);
        }
        lookback_publish(a.tile_state, tile, 4ull + cs, lane);
        const uint32_t nxt = grab_tile(a.tile_counter, lane);
        if (ptile != ~0u) place_staged(a, ptile, slot1, pcs, tmp, bar, parity, lane);
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
    if (ptile != ~0u) place_staged(a, ptile, slot1, pcs, tmp, bar, parity, lane);
}

}  // namespace bsg
