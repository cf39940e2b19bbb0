// Batched codec: many independent chunks (uneven sizes, element sizes 1, 2,
// 4 or 8, their own block sizes) compressed or decompressed by ONE persistent
// launch.  Sec. 4.2.1 makes blocks independent units of work; here the work
// queue runs over every (chunk, block) item of the batch, so the GPU stays
// full however the sizes are spread.
//
// Host side: bsgpu_batch_plan() validates the chunks and writes a table image
// (one record per chunk, then the first item index of every chunk); the
// caller copies it to device memory, where the kernels read it.  Each chunk's
// blocks are numbered locally: its look-back state, block index and status
// start at its own first item, so a chunk's stream is exactly the one
// bsgpu_compress() writes for it alone.
#include <cuda_runtime.h>

#include <cstring>

#include "../../include/bsgpu.h"
#include "codec.cuh"

#include <nvtx3/nvToolsExt.h>

namespace {
// An NVTX range around a C-ABI call, so that a profiler's timeline shows
// the library's entry points (header-only NVTX: without a tool attached
// each push and pop is a check of a null callback).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace bsg {

// One chunk as the kernels see it (80 bytes, written by the planner).
struct BatchChunk {
    const uint8_t *in;
    uint8_t *out;
    uint64_t n_elem;
    uint64_t in_bytes;   // decompress: stream length
    uint64_t out_cap;    // compress: capacity of out
    uint64_t item0;      // first item of the chunk
    uint32_t es, B, nb, last_B;
    uint32_t tail, pad0;
    uint64_t *offs;      // the chunk's own block index, or null (batch-wide array)
};
static_assert(sizeof(BatchChunk) == 80, "table record layout");

struct BatchArgs {
    const BatchChunk *chunks;
    const uint64_t *starts;       // n_chunks + 1 first-item indices
    uint32_t n_chunks;
    uint32_t n_items;
    uint64_t *state;              // compress: look-back state, one per item
    uint32_t *counter;            // work-queue counter
    uint8_t *slots;               // compress: two staging slots per CTA
    uint64_t *out_bytes;          // compress: per chunk stream length
    const uint64_t *in_bytes;     // decompress: per chunk stream length, or null
    uint64_t *offsets;            // per item block offsets, or null
    int *status;                  // per chunk status
    int level;
};

// Chunk holding item t: the last c with starts[c] <= t (every chunk has at
// least one item, so the starts are strictly increasing).
BSG_D uint32_t find_chunk(const uint64_t *starts, uint32_t n, uint32_t t)
{
    uint32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (__ldg(starts + mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The single-stream argument block of chunk c (local block numbering).
BSG_D CodecArgs chunk_args(const BatchArgs &b, uint32_t c)
{
    const BatchChunk &ch = b.chunks[c];
    CodecArgs a{};
    a.in = ch.in;
    a.out = ch.out;
    a.in_bytes = b.in_bytes ? b.in_bytes[c] : ch.in_bytes;
    a.out_cap = ch.out_cap;
    a.out_bytes = b.out_bytes ? b.out_bytes + c : nullptr;
    a.block_offsets = ch.offs ? ch.offs : (b.offsets ? b.offsets + ch.item0 : nullptr);
    a.tile_state = b.state ? b.state + ch.item0 : nullptr;
    a.status = b.status + c;
    a.n_elem = ch.n_elem;
    a.es = ch.es;
    a.B = ch.B;
    a.nb = ch.nb;
    a.last_B = ch.last_B;
    a.tail_elems = ch.tail;
    a.level = b.level;
    return a;
}

// A chunk of fewer than 8 elements: header plus the elements verbatim.
BSG_D void compress_tiny(const CodecArgs &a, uint32_t lane)
{
    const uint32_t tb = a.tail_elems * a.es;
    if (12 + tb > a.out_cap) {
        if (lane == 0) set_status(a.status, BSGPU_ERR_SPACE);
        return;
    }
    write_chunk_header(a.out, a.n_elem * a.es, a.B * a.es, lane);
    for (uint32_t k = lane; k < tb; k += 32) a.out[12 + k] = a.in[k];
    if (lane == 0) *a.out_bytes = 12 + tb;
}

// Bit-transpose block `tile` of chunk `ch` into `tmp`: in place through
// registers after a bulk copy when the shape allows, else straight from
// global memory by the byte-wise path (a chunk's shortened last block).
// The in-place transposes as calls of their own, so that each is
// register-allocated alone rather than all three inside one kernel.
__device__ __noinline__ void batch_shuffle2(uint8_t *tmp, uint32_t Bb, uint32_t lane)
{
    shuffle2_inplace(tmp, Bb, lane);
}
__device__ __noinline__ void batch_shuffle4(uint8_t *tmp, uint32_t Bb, uint32_t lane)
{
    shuffle4_inplace(tmp, Bb, lane, NoRound{});
}
__device__ __noinline__ void batch_shuffle8(uint8_t *tmp, uint32_t Bb, uint32_t lane)
{
    shuffle8_inplace(tmp, Bb, lane);
}

BSG_D void batch_prepare(const BatchChunk &ch, uint32_t tile, uint32_t Bb, uint8_t *tmp,
                         uint64_t *bar, uint32_t &parity, int *status, uint32_t lane)
{
    const uint32_t es = ch.es;
    const uint8_t *src = ch.in + (uint64_t)tile * ch.B * es;
    if (!shuffle_inplace_ok(es, Bb)) {
        // rare (a chunk's shortened last block): the byte-wise path keeps
        // register pressure down
        shuffle_generic(src, tmp, Bb, es, lane);
        __syncwarp();
        return;
    }
    if (load_block(tmp, src, Bb * es, bar, lane)) {
        if (!mbar_wait_bounded(bar, parity) && lane == 0) set_status(status, BSGPU_ERR_TIMEOUT);
        parity ^= 1u;
    }
    if (es == 2)
        batch_shuffle2(tmp, Bb, lane);
    else if (es == 4)
        batch_shuffle4(tmp, Bb, lane);
    else
        batch_shuffle8(tmp, Bb, lane);
    __syncwarp();
}

// Exclusive prefix of block `tile` of chunk c by look-back, then its
// placement (index entry, chunk header, verbatim tail, stream length); the
// staging slot's lines are then dropped from L2.
BSG_D void batch_place(const BatchArgs &b, uint32_t c, uint32_t tile, const uint8_t *slot,
                       uint32_t cs, uint8_t *buf, uint64_t *bar, uint32_t &parity, uint32_t lane)
{
    const CodecArgs a = chunk_args(b, c);
    // the staged bytes come back into the warp's free block buffer by one
    // bulk copy while the look-back finds the block's offset
    const uint32_t bytes = r16(4 + cs);
    fence_proxy_async_all();
    __syncwarp();
    if (lane == 0) {
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(buf, slot, bytes, bar);
    }
    const uint64_t excl = lookback_resolve(a.tile_state, tile, 4ull + cs, a.status, lane);
    if (!mbar_wait_bounded(bar, parity) && lane == 0) set_status(a.status, BSGPU_ERR_TIMEOUT);
    parity ^= 1u;
    compress_place(a, tile, buf, cs, 12 + excl, lane);
    __syncwarp();
    discard_slot(slot, 4 + cs, lane);
}

// Shared memory of one warp of the batch kernels, rounded up so that the
// warps of a multi-warp CTA each get a 128-byte aligned slice.
template <int LEVEL>
__host__ __device__ constexpr uint32_t batch_compress_warp_smem() { return r128(FastPlan<LEVEL>::BYTES); }
__host__ __device__ constexpr uint32_t batch_decompress_warp_smem() { return r128(INPLACE_BUF + 16); }

// Persistent, one shared buffer per warp (as compress_fast_kernel): per
// item, transpose the block, LZ4-encode it into this warp's staging slot,
// publish its size in its chunk's look-back state, then place the PREVIOUS
// item's block, whose predecessors have long published theirs.  Only the
// chunk index and local block number live across an item; the chunk's
// fields are re-read from its (cached) table record where they are used.
// A CTA holds 1, 2 or 4 warps (a launch-shape choice of the autotuner); they
// share nothing but the CTA: each warp has its own slice of the dynamic
// shared memory, its own barrier and staging slots, and takes its own items.
template <int LEVEL, int W>
__global__ void __launch_bounds__(32 * W, 20 / W) compress_batch_kernel(const __grid_constant__ BatchArgs b)
{
    using L = FastPlan<LEVEL>;
    // a staged block comes back into the buffer and the encoder's scratch
    // after it (both free by then) for its placement
    static_assert(L::TMP + L::SCR >= r16(4 + lz4b(L::MAXB)), "placement buffer");
    extern __shared__ __align__(128) uint8_t smem_all[];
    const uint32_t warp = W == 1 ? 0u : threadIdx.x >> 5;
    uint8_t *sm = smem_all + (size_t)warp * batch_compress_warp_smem<LEVEL>();
    uint8_t *tmp = sm;
    void *scratch = sm + L::TMP;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::TMP + r16(L::SCR));
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const uint32_t gw = blockIdx.x * W + warp;   // this warp's slot pair
    uint8_t *slot0 = b.slots + (size_t)(2 * gw) * FAST_SLOT_BYTES;
    uint8_t *slot1 = slot0 + FAST_SLOT_BYTES;
    uint32_t parity = 0;
    uint32_t ptile = ~0u, pchunk = 0, pcs = 0;  // the block waiting to be placed, in slot1
    uint32_t t = grab_tile(b.counter, lane);
    while (t < b.n_items) {
        const uint32_t c = find_chunk(b.starts, b.n_chunks, t);
        const BatchChunk &ch = b.chunks[c];
        const uint32_t tile = t - (uint32_t)ch.item0;
        const uint32_t nb = ch.nb;
        uint32_t cs = 0;
        if (nb == 0) {
            compress_tiny(chunk_args(b, c), lane);
        } else {
            const uint32_t Bb = tile + 1 == nb ? ch.last_B : ch.B;
            const uint32_t S = Bb * ch.es;
            batch_prepare(ch, tile, Bb, tmp, bar, parity, b.status + c, lane);
            // bit-rows are Bb/8 bytes long: the previous row is one of the candidates
            if (LEVEL >= 1)
                cs = lz4_encode_warp<1, L::HBITS>(tmp, S, Bb / 8, slot0 + 4,
                                                  static_cast<uint16_t *>(scratch));
            else if (S % 128u == 0)
                cs = lz4_encode_bitmap_fast(tmp, S, Bb / 8, slot0 + 4,
                                            static_cast<uint32_t *>(scratch));
            else
                cs = lz4_encode_bitmap(tmp, S, Bb / 8, slot0 + 4, static_cast<uint32_t *>(scratch));
            if (cs == 0xffffffffu) {  // progress guard (not reachable for valid sizes)
                if (lane == 0) set_status(b.status + c, BSGPU_ERR_CUDA);
                cs = 0;
            }
            if (lane == 0) put_be32(slot0, cs);
            __syncwarp();
            lookback_publish(b.state + ch.item0, tile, 4ull + cs, lane);
        }
        const uint32_t nxt = grab_tile(b.counter, lane);
        if (ptile != ~0u) batch_place(b, pchunk, ptile, slot1, pcs, tmp, bar, parity, lane);
        __syncwarp();
        if (nb != 0) {
            ptile = tile;
            pchunk = c;
            pcs = cs;
            uint8_t *x = slot0;
            slot0 = slot1;
            slot1 = x;
        } else {
            ptile = ~0u;
        }
        t = nxt;
        // the next load overwrites `tmp`: the async proxy follows the generic reads
        fence_proxy_async_smem();
        __syncwarp();
    }
    if (ptile != ~0u) batch_place(b, pchunk, ptile, slot1, pcs, tmp, bar, parity, lane);
}

// Header of a chunk's stream (checked with its first item).
BSG_D void check_header(const CodecArgs &a, uint32_t lane)
{
    uint32_t ok = 1;
    if (lane < 12) {
        const uint8_t want = lane < 8 ? (uint8_t)((a.n_elem * a.es) >> (8 * (7 - lane)))
                                      : (uint8_t)(((uint64_t)a.B * a.es) >> (8 * (11 - lane)));
        ok = a.in_bytes >= 12 && a.in[lane] == want;
    }
    if (__ballot_sync(FULL, !ok) && lane == 0) set_status(a.status, BSGPU_ERR_CORRUPT);
}

// The verbatim tail after a chunk's last block, or after the header alone for
// a chunk without blocks (whose stream is then exactly 12 + tail bytes).
BSG_D void copy_tail(const CodecArgs &a, uint32_t lane)
{
    const uint32_t tb = a.tail_elems * a.es;
    const uint64_t first = (a.n_elem - a.tail_elems) * a.es;
    const bool ok = a.nb ? a.in_bytes >= 12 + tb : a.in_bytes == 12 + tb;
    if (ok)
        for (uint32_t k = lane; k < tb; k += 32) a.out[first + k] = a.in[a.in_bytes - tb + k];
    else if (lane == 0)
        set_status(a.status, BSGPU_ERR_CORRUPT);
}

// Start fetching item t's stream bytes into the end of the buffer `comp`
// (nothing for a chunk without blocks).
BSG_D DecLoad batch_issue(const BatchArgs &b, uint32_t c, uint32_t t, uint8_t *comp,
                          uint64_t *bar, uint32_t lane)
{
    const CodecArgs a = chunk_args(b, c);
    if (a.nb == 0) return DecLoad{};
    return dec_issue(a, t - (uint32_t)b.chunks[c].item0, comp, bar, lane, INPLACE_BUF);
}

// LZ4-decode block `tile` of chunk c (stream bytes in `comp`) into `dec`;
// true when it decoded to exactly its size.
BSG_D bool batch_decode(const BatchArgs &b, uint32_t c, uint32_t tile, const DecLoad &cur,
                        uint8_t *comp, uint8_t *dec, uint32_t lane)
{
    const BatchChunk &ch = b.chunks[c];
    const uint32_t Bb = tile + 1 == ch.nb ? ch.last_B : ch.B;
    bool good = cur.ok;
    if (good) {
        if (cur.eidx != ~0u) comp[cur.eidx] = cur.ebyte;
        __syncwarp();
        good = get_be32(comp + cur.delta) == cur.clen &&
               lz4_decode_warp(comp, cur.delta + 4, cur.clen, dec, Bb * ch.es) == 0;
    }
    if (!good && lane == 0) set_status(b.status + c, BSGPU_ERR_CORRUPT);
    return good;
}

// The in-place un-transposes as calls of their own, so that each is
// register-allocated alone rather than all three inside one kernel.
__device__ __noinline__ void batch_unshuffle2(uint8_t *buf, uint32_t Bb, uint32_t lane)
{
    unshuffle2_inplace(buf, Bb, lane);
}
__device__ __noinline__ void batch_unshuffle4(uint8_t *buf, uint32_t Bb, uint32_t lane)
{
    unshuffle4_inplace(buf, Bb, lane);
}
__device__ __noinline__ void batch_unshuffle8(uint8_t *buf, uint32_t Bb, uint32_t lane)
{
    unshuffle8_inplace(buf, Bb, lane);
}

// Persistent, one shared buffer per warp decoded in place (as
// decompress_inplace_kernel): per item, wait for its stream bytes, LZ4-decode,
// un-transpose and store, then fetch the next item's bytes (of whichever chunk
// it belongs to) once the store has read the buffer.  As in the compressor
// only chunk indices and block numbers live across an item, and a CTA holds 1,
// 2 or 4 independent warps, each with its own slice of shared memory.
template <int W>
__global__ void __launch_bounds__(32 * W, 20 / W) decompress_batch_kernel(const __grid_constant__ BatchArgs b)
{
    extern __shared__ __align__(128) uint8_t smem_all[];
    uint8_t *sm = smem_all + (W == 1 ? 0u : (threadIdx.x >> 5) * batch_decompress_warp_smem());
    uint8_t *buf = sm;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + INPLACE_BUF);
    const uint32_t lane = threadIdx.x & 31u;
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;
    uint32_t t = grab_tile(b.counter, lane);
    uint32_t c = 0;
    DecLoad ld{};
    if (t < b.n_items) {
        c = find_chunk(b.starts, b.n_chunks, t);
        ld = batch_issue(b, c, t, buf, bar, lane);
    }
    while (t < b.n_items) {
        const uint32_t tile = t - (uint32_t)b.chunks[c].item0;
        const uint32_t nb = b.chunks[c].nb;
        const DecLoad cur = ld;
        if (cur.bulk) {
            if (!mbar_wait_bounded(bar, parity) && lane == 0) set_status(b.status + c, BSGPU_ERR_TIMEOUT);
            parity ^= 1u;
        }
        if (tile == 0) check_header(chunk_args(b, c), lane);
        const uint32_t nxt = grab_tile(b.counter, lane);
        const uint32_t nc = nxt < b.n_items ? find_chunk(b.starts, b.n_chunks, nxt) : c;
        if (nb) {
            const bool good = batch_decode(b, c, tile, cur, buf + cur.off, buf, lane);
            __syncwarp();
            const BatchChunk &ch = b.chunks[c];
            const uint32_t es = ch.es;
            const uint32_t Bb = tile + 1 == nb ? ch.last_B : ch.B;
            const uint32_t S = Bb * es;
            uint8_t *dst = ch.out + (uint64_t)tile * ch.B * es;
            if (good && unshuffle_inplace_ok(es, Bb)) {
                if (es == 2)
                    batch_unshuffle2(buf, Bb, lane);
                else if (es == 4)
                    batch_unshuffle4(buf, Bb, lane);
                else
                    batch_unshuffle8(buf, Bb, lane);
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
                unshuffle_generic(buf, dst, Bb, es, lane);  // 1-byte elements, a shortened block
            }
        }
        if (nb == 0 || tile + 1 == nb) copy_tail(chunk_args(b, c), lane);
        __syncwarp();
        // the next item's bytes go into the same buffer once the store has read it
        if (lane == 0) bulk_wait_read0();
        __syncwarp();
        ld = DecLoad{};
        if (nxt < b.n_items) {
            fence_proxy_async_smem();
            __syncwarp();
            ld = batch_issue(b, nc, nxt, buf, bar, lane);
        }
        t = nxt;
        c = nc;
    }
    if (lane == 0) bulk_wait0();
    __syncwarp();
}

// Block offsets of every chunk without its own index by walking its chain of
// length fields: one warp per chunk, the chunk's stream staged through
// shared memory (chain_walk_staged).
__global__ void __launch_bounds__(32, 1) chain_walk_batch_kernel(const __grid_constant__ BatchArgs b)
{
    extern __shared__ __align__(128) uint8_t sm[];
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t c = blockIdx.x; c < b.n_chunks; c += gridDim.x) {
        if (b.chunks[c].offs) continue;   // a chunk with its own index
        const CodecArgs a = chunk_args(b, c);
        if (a.nb == 0) continue;
        bool timely = true;
        const bool ok = chain_walk_staged(a.in, a.in_bytes, a.nb, (uint64_t)a.tail_elems * a.es,
                                          a.block_offsets, sm, lane, timely);
        if (lane == 0 && !timely) set_status(a.status, BSGPU_ERR_TIMEOUT);
        else if (lane == 0 && !ok) set_status(a.status, BSGPU_ERR_CORRUPT);
        __syncwarp();
    }
}

}  // namespace bsg

using namespace bsg;

namespace {

constexpr size_t BATCH_HEADER = 256;  // [0] unused status word, [4] work-queue counter

size_t r256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t table_bytes(uint32_t n) { return ((size_t)n * sizeof(BatchChunk) + 8ull * (n + 1) + 15) & ~(size_t)15; }

struct BatchWs {
    size_t state, slots, offsets, total;
};

BatchWs batch_ws(int op, uint64_t n_items, uint32_t grid_max)
{
    BatchWs w{};
    size_t o = BATCH_HEADER;
    if (op == BSGPU_OP_COMPRESS) {
        w.state = o;
        o += r256(8 * n_items);
        w.slots = o;
        o += (size_t)grid_max * 2 * FAST_SLOT_BYTES;
    } else {
        w.offsets = o;  // block offsets when the caller has no index
        o += r256(8 * n_items);
    }
    w.total = o;
    return w;
}

int sm_count()
{
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Resident CTAs of `warps` warps per SM (at least 1).
template <typename K>
uint32_t occupancy(K kernel, uint32_t smem, uint32_t warps)
{
    int n = 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, (int)(32 * warps), smem) !=
            cudaSuccess || n < 1)
        n = 1;
    return (uint32_t)n;
}

template <typename K>
cudaError_t launch_batch(K kernel, uint32_t smem, uint32_t grid, uint32_t warps, cudaStream_t s,
                         const BatchArgs &b)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    kernel<<<grid, 32 * warps, smem, s>>>(b);
    return cudaGetLastError();
}

// Persistent grid of CTAs of `warps` warps: ctas_per_sm (0 = as many as fit)
// on every SM, never more warps than the items or the staging slots.
uint32_t batch_grid(uint32_t fit, uint32_t ctas_per_sm, uint32_t warps, uint64_t n_items)
{
    uint32_t per = ctas_per_sm && ctas_per_sm < fit ? ctas_per_sm : fit;
    uint64_t g = (uint64_t)sm_count() * per;
    if (g * warps > FAST_MAX_WARPS) g = FAST_MAX_WARPS / warps;
    const uint64_t need = (n_items + warps - 1) / warps;
    if (g > need) g = need;
    return g ? (uint32_t)g : 1u;
}

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; }

template <int LEVEL, int W>
cudaError_t launch_compress_batch(const BatchArgs &b, uint32_t ctas_per_sm, uint64_t n_items,
                                  cudaStream_t s)
{
    const uint32_t smem = W * batch_compress_warp_smem<LEVEL>();
    const uint32_t g = batch_grid(occupancy(compress_batch_kernel<LEVEL, W>, smem, W), ctas_per_sm,
                                  W, n_items);
    return launch_batch(compress_batch_kernel<LEVEL, W>, smem, g, W, s, b);
}

template <int W>
cudaError_t launch_decompress_batch(const BatchArgs &b, uint32_t ctas_per_sm, uint64_t n_items,
                                    cudaStream_t s)
{
    const uint32_t smem = W * batch_decompress_warp_smem();
    const uint32_t g = batch_grid(occupancy(decompress_batch_kernel<W>, smem, W), ctas_per_sm, W,
                                  n_items);
    return launch_batch(decompress_batch_kernel<W>, smem, g, W, s, b);
}

}  // namespace

extern "C" {

size_t bsgpu_batch_table_bytes(uint32_t n_chunks)
{
    return n_chunks ? table_bytes(n_chunks) : 0;
}

int bsgpu_batch_plan(int op, const bsgpu_chunk *chunks, uint32_t n_chunks, void *table,
                     size_t table_bytes_given, uint64_t *n_items, size_t *ws_bytes)
{
    if (op != BSGPU_OP_COMPRESS && op != BSGPU_OP_DECOMPRESS) return BSGPU_ERR_ARG;
    if (!chunks || !n_chunks || !table || !n_items || !ws_bytes) return BSGPU_ERR_ARG;
    if (table_bytes_given < table_bytes(n_chunks)) return BSGPU_ERR_SPACE;
    BatchChunk *rec = static_cast<BatchChunk *>(table);
    uint64_t *starts = reinterpret_cast<uint64_t *>(rec + n_chunks);
    uint64_t items = 0;
    for (uint32_t c = 0; c < n_chunks; c++) {
        const bsgpu_chunk &k = chunks[c];
        const uint64_t es = k.elem_size;
        if (es != 1 && es != 2 && es != 4 && es != 8) return BSGPU_ERR_ARG;
        const uint64_t B = k.block_elems ? k.block_elems : 4096 / es;
        if (B == 0 || B % 8 || B * es > 8192) return BSGPU_ERR_ARG;
        if ((!k.in && k.n_elem) || (!k.out && (op == BSGPU_OP_COMPRESS || k.n_elem)))
            return BSGPU_ERR_ARG;
        if ((k.in && !aligned(k.in, 16)) || (k.out && !aligned(k.out, 16)) ||
            !aligned(k.block_offsets, 8))
            return BSGPU_ERR_ALIGN;
        const uint64_t full = k.n_elem / B, rem = k.n_elem % B, last = rem - rem % 8;
        const uint64_t nb = full + (last ? 1 : 0);
        if (op == BSGPU_OP_COMPRESS &&
            k.out_cap < bsgpu_compress_bound(k.n_elem, k.elem_size, (size_t)B))
            return BSGPU_ERR_SPACE;
        if (op == BSGPU_OP_DECOMPRESS && !k.in) return BSGPU_ERR_ARG;
        BatchChunk r{};
        r.in = static_cast<const uint8_t *>(k.in);
        r.out = static_cast<uint8_t *>(k.out);
        r.n_elem = k.n_elem;
        r.in_bytes = k.in_bytes;
        r.out_cap = k.out_cap;
        r.item0 = items;
        r.es = (uint32_t)es;
        r.B = (uint32_t)B;
        r.nb = (uint32_t)nb;
        r.last_B = (uint32_t)(last ? last : B);
        r.tail = (uint32_t)(rem % 8);
        r.offs = k.block_offsets;
        std::memcpy(rec + c, &r, sizeof r);
        starts[c] = items;
        items += nb ? nb : 1;  // a chunk without blocks still takes one item
        if (items >= (1ull << 31)) return BSGPU_ERR_ARG;
    }
    starts[n_chunks] = items;
    *n_items = items;
    *ws_bytes = batch_ws(op, items, FAST_MAX_WARPS).total;
    return BSGPU_OK;
}

int bsgpu_compress_batch_ex(const void *d_table, uint32_t n_chunks, uint64_t n_items, int level,
                            uint64_t *d_out_bytes, uint64_t *d_block_offsets, int *d_chunk_status,
                            void *ws, size_t ws_bytes, uint32_t ctas_per_sm,
                            uint32_t warps_per_cta, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_compress_batch_ex");
    if (!d_table || !n_chunks || !n_items || n_items >= (1ull << 31) || level < 0 || level > 1)
        return BSGPU_ERR_ARG;
    if (warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4) return BSGPU_ERR_ARG;
    if (!d_out_bytes || !d_chunk_status || !ws) return BSGPU_ERR_ARG;
    if (!aligned(d_table, 16) || !aligned(ws, 16) || !aligned(d_out_bytes, 8) ||
        !aligned(d_block_offsets, 8) || !aligned(d_chunk_status, 4))
        return BSGPU_ERR_ALIGN;
    const BatchWs w = batch_ws(BSGPU_OP_COMPRESS, n_items, FAST_MAX_WARPS);
    if (ws_bytes < w.total) return BSGPU_ERR_SPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws, 0, w.state + 8 * n_items, s) != cudaSuccess ||
        cudaMemsetAsync(d_chunk_status, 0, sizeof(int) * n_chunks, s) != cudaSuccess)
        return BSGPU_ERR_CUDA;
    BatchArgs b{};
    b.chunks = static_cast<const BatchChunk *>(d_table);
    b.starts = reinterpret_cast<const uint64_t *>(b.chunks + n_chunks);
    b.n_chunks = n_chunks;
    b.n_items = (uint32_t)n_items;
    b.state = reinterpret_cast<uint64_t *>((uint8_t *)ws + w.state);
    b.counter = reinterpret_cast<uint32_t *>((uint8_t *)ws + 4);
    b.slots = (uint8_t *)ws + w.slots;
    b.out_bytes = d_out_bytes;
    b.offsets = d_block_offsets;
    b.status = d_chunk_status;
    b.level = level;
    cudaError_t e;
    switch (warps_per_cta * 2 + (level >= 1 ? 1 : 0)) {
    case 2: e = launch_compress_batch<0, 1>(b, ctas_per_sm, n_items, s); break;
    case 3: e = launch_compress_batch<1, 1>(b, ctas_per_sm, n_items, s); break;
    case 4: e = launch_compress_batch<0, 2>(b, ctas_per_sm, n_items, s); break;
    case 5: e = launch_compress_batch<1, 2>(b, ctas_per_sm, n_items, s); break;
    case 8: e = launch_compress_batch<0, 4>(b, ctas_per_sm, n_items, s); break;
    case 9: e = launch_compress_batch<1, 4>(b, ctas_per_sm, n_items, s); break;
    default: return BSGPU_ERR_ARG;   // 3 warps per CTA: not built
    }
    return e == cudaSuccess ? BSGPU_OK : BSGPU_ERR_CUDA;
}

int bsgpu_compress_batch(const void *d_table, uint32_t n_chunks, uint64_t n_items, int level,
                         uint64_t *d_out_bytes, uint64_t *d_block_offsets, int *d_chunk_status,
                         void *ws, size_t ws_bytes, uint32_t ctas_per_sm, void *stream)
{
    return bsgpu_compress_batch_ex(d_table, n_chunks, n_items, level, d_out_bytes,
                                   d_block_offsets, d_chunk_status, ws, ws_bytes, ctas_per_sm, 1,
                                   stream);
}

int bsgpu_decompress_batch_ex(const void *d_table, uint32_t n_chunks, uint64_t n_items,
                              const uint64_t *d_in_bytes, const uint64_t *d_block_offsets,
                              int *d_chunk_status, void *ws, size_t ws_bytes,
                              uint32_t ctas_per_sm, uint32_t warps_per_cta, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_decompress_batch_ex");
    if (!d_table || !n_chunks || !n_items || n_items >= (1ull << 31)) return BSGPU_ERR_ARG;
    if (warps_per_cta != 1 && warps_per_cta != 2 && warps_per_cta != 4) return BSGPU_ERR_ARG;
    if (!d_chunk_status || !ws) return BSGPU_ERR_ARG;
    if (!aligned(d_table, 16) || !aligned(ws, 16) || !aligned(d_in_bytes, 8) ||
        !aligned(d_block_offsets, 8) || !aligned(d_chunk_status, 4))
        return BSGPU_ERR_ALIGN;
    const BatchWs w = batch_ws(BSGPU_OP_DECOMPRESS, n_items, FAST_MAX_WARPS);
    if (ws_bytes < w.total) return BSGPU_ERR_SPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws, 0, BATCH_HEADER, s) != cudaSuccess ||
        cudaMemsetAsync(d_chunk_status, 0, sizeof(int) * n_chunks, s) != cudaSuccess)
        return BSGPU_ERR_CUDA;
    BatchArgs b{};
    b.chunks = static_cast<const BatchChunk *>(d_table);
    b.starts = reinterpret_cast<const uint64_t *>(b.chunks + n_chunks);
    b.n_chunks = n_chunks;
    b.n_items = (uint32_t)n_items;
    b.counter = reinterpret_cast<uint32_t *>((uint8_t *)ws + 4);
    b.in_bytes = d_in_bytes;
    b.status = d_chunk_status;
    if (d_block_offsets) {
        b.offsets = const_cast<uint64_t *>(d_block_offsets);
    } else {
        b.offsets = reinterpret_cast<uint64_t *>((uint8_t *)ws + w.offsets);
        if (cudaFuncSetAttribute(chain_walk_batch_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)WALK_SMEM) != cudaSuccess)
            return BSGPU_ERR_CUDA;
        const uint32_t g = (uint32_t)(n_chunks < (uint32_t)sm_count() ? n_chunks : sm_count());
        chain_walk_batch_kernel<<<g, 32, WALK_SMEM, s>>>(b);
        if (cudaGetLastError() != cudaSuccess) return BSGPU_ERR_CUDA;
    }
    cudaError_t e;
    switch (warps_per_cta) {
    case 1: e = launch_decompress_batch<1>(b, ctas_per_sm, n_items, s); break;
    case 2: e = launch_decompress_batch<2>(b, ctas_per_sm, n_items, s); break;
    case 4: e = launch_decompress_batch<4>(b, ctas_per_sm, n_items, s); break;
    default: return BSGPU_ERR_ARG;   // 3 warps per CTA: not built
    }
    return e == cudaSuccess ? BSGPU_OK : BSGPU_ERR_CUDA;
}

int bsgpu_decompress_batch(const void *d_table, uint32_t n_chunks, uint64_t n_items,
                           const uint64_t *d_in_bytes, const uint64_t *d_block_offsets,
                           int *d_chunk_status, void *ws, size_t ws_bytes, uint32_t ctas_per_sm,
                           void *stream)
{
    return bsgpu_decompress_batch_ex(d_table, n_chunks, n_items, d_in_bytes, d_block_offsets,
                                     d_chunk_status, ws, ws_bytes, ctas_per_sm, 1, stream);
}

}  // extern "C"
