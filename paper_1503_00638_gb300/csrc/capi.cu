// C-ABI of libbsgpu (declared in include/bsgpu.h): argument checks,
// workspace layout, grid sizing and kernel launches.  Nothing here allocates.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/bsgpu.h"
#include "kernels.cuh"
#include "shuffle.cuh"

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

using namespace bsg;

namespace {

constexpr size_t WS_HEADER = 256;  // int status, uint32 tile counter, padding
constexpr uint64_t MAX_BLOCK_BYTES = 65536;

inline size_t r256(size_t x) { return (x + 255) & ~size_t(255); }

inline bool es_ok(size_t es) { return es == 1 || es == 2 || es == 4 || es == 8; }

struct Geometry {
    uint64_t n;        // elements
    uint32_t es, B;    // element size, block elements
    uint32_t nb;       // blocks (full + shortened last)
    uint32_t last_B;   // elements of the last block
    uint32_t tail;     // trailing elements copied verbatim (< 8)
};

// Blocks of B elements (0 = 4096 bytes, Sec. 4.2.1); a shortened last block
// of the remaining elements rounded down to a multiple of 8; the rest verbatim.
int geometry(size_t n, size_t es, size_t block_elems, Geometry &g)
{
    if (!es_ok(es)) return BSGPU_ERR_ARG;
    size_t B = block_elems ? block_elems : 4096 / es;
    if (B == 0 || B % 8 != 0 || B * es > MAX_BLOCK_BYTES) return BSGPU_ERR_ARG;
    uint64_t full = n / B, rem = n % B, last = rem - rem % 8;
    uint64_t nb = full + (last ? 1 : 0);
    if (nb >= (1ull << 31)) return BSGPU_ERR_ARG;
    g.n = n;
    g.es = (uint32_t)es;
    g.B = (uint32_t)B;
    g.nb = (uint32_t)nb;
    g.last_B = (uint32_t)(last ? last : B);
    g.tail = (uint32_t)(rem % 8);
    return BSGPU_OK;
}

uint64_t stream_bound(const Geometry &g)
{
    auto lz = [](uint64_t s) { return s + s / 255 + 16; };
    uint64_t full = g.nb - (g.last_B != g.B ? 1 : 0);
    uint64_t b = 12 + full * (4 + lz((uint64_t)g.B * g.es));
    if (g.last_B != g.B && g.nb) b += 4 + lz((uint64_t)g.last_B * g.es);
    return b + (uint64_t)g.tail * g.es;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Persistent grid: warp-CTAs resident on all SMs, never more than the work.
uint32_t persistent_grid(uint32_t smem_per_cta, uint64_t work)
{
    int dev = 0, sms = 148, smem_sm = 228 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
    uint32_t per_sm = (uint32_t)(smem_sm / (smem_per_cta + 1024));
    if (per_sm > 32) per_sm = 32;
    if (per_sm == 0) per_sm = 1;
    uint64_t grid = (uint64_t)sms * per_sm;
    if (grid > work) grid = work;
    return grid ? (uint32_t)grid : 1u;
}

struct WsLayout {
    size_t state, autos, pairs, cft, qtab, offsets, segs, slots, gslots, total;
    uint32_t gslot_warps;  // warps the general compressor's slots cover
};

// SMs the general compressor's staging slots are sized for (at least the
// device's count; GB300 has 152)
constexpr uint32_t GEN_MAX_SMS = 160;

// What the flags of the visibility entry points add to the workspace.
struct VisOpts {
    bool tslow = false, full = false;
    size_t n_ft = 0;                    // compensated c per (freq, time)
    size_t qtab_bytes = 0;
};

VisOpts vis_opts(int flags, int64_t n_freq, int64_t n_in, int64_t n_time)
{
    VisOpts o;
    o.tslow = (flags & BSGPU_VIS_TIME_SLOWEST) != 0;
    o.full = (flags & BSGPU_VIS_FULL_COV) != 0;
    if (flags & BSGPU_VIS_COMPENSATE) o.n_ft = (size_t)n_freq * n_time;
    if (o.full) {
        const uint64_t ft = (uint64_t)n_freq * n_time, M = (uint64_t)n_in * n_in;
        o.qtab_bytes = ft * M * 4;
    }
    return o;
}

// Whether compress takes the fast kernel: full blocks of at most 8 KiB of 2-,
// 4- or 8-byte elements (a cube in any order, any time axis).
bool fast_shape(const Geometry &g)
{
    return shuffle_inplace_ok(g.es, g.B);
}

// n_ft: entries of the per-(freq, time) compensated-c table (0 = none)
WsLayout ws_layout(int op, const Geometry &g, size_t n_auto, size_t n_prod, uint64_t n_time = 0,
                   const VisOpts &opts = VisOpts())
{
    WsLayout L{};
    size_t o = WS_HEADER;
    if (op == BSGPU_OP_COMPRESS || op == BSGPU_OP_COMPRESS_VIS) {
        L.state = o;
        o += r256((size_t)g.nb * 8);
        if (g.nb && fast_shape(g)) {
            L.slots = o;
            o += (size_t)FAST_MAX_WARPS * 2 * FAST_SLOT_BYTES;
        }
        // the general compressor's staging slots: for its one shortened last
        // block after the fast path, else for as many warps as can be
        // resident (at most GEN_MAX_SMS SMs)
        const uint32_t gwork = !g.nb ? 0u : fast_shape(g) ? (g.last_B != g.B ? 1u : 0u) : g.nb;
        if (gwork) {
            const uint32_t maxb = maxb_class(g.B * g.es);
            const uint32_t smem = compress_smem_bytes(maxb, 0, true);
            uint32_t per_sm = (228u * 1024u) / (smem + 1024u);
            if (per_sm == 0) per_sm = 1;
            uint64_t w = (uint64_t)GEN_MAX_SMS * per_sm;
            if (w > gwork) w = gwork;
            L.gslots = o;
            L.gslot_warps = (uint32_t)w;
            o += r256((size_t)w * 2 * compress_slot_bytes(maxb));
        }
    }
    if (op == BSGPU_OP_COMPRESS_VIS || op == BSGPU_OP_REDUCE_PRECISION) {
        L.autos = o;
        o += r256(n_auto * 4);
        L.pairs = o;
        o += r256(n_prod * 4);
        if (opts.n_ft) {
            L.cft = o;
            o += r256(opts.n_ft * 4);
        }
        if (opts.full) {
            L.qtab = o;
            o += r256(opts.qtab_bytes);
        }
    }
    if (op == BSGPU_OP_DECOMPRESS) {
        L.offsets = o;
        o += r256((size_t)g.nb * 8);
        L.segs = o;   // the parallel recovery of a missing block index
        o += r256(SEG_WS_BYTES);
    }
    L.total = o;
    return L;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? BSGPU_OK : BSGPU_ERR_CUDA; }

// Cube geometry checks shared by the visibility entry points.
int vis_check(int64_t n_freq, int64_t n_in, int64_t n_time, double N, double f, uint64_t &n_prod,
              uint64_t &n_cplx)
{
    if (n_freq <= 0 || n_in <= 0 || n_time <= 0 || n_in > 65535) return BSGPU_ERR_ARG;
    if (!(N > 0) || !std::isfinite(N) || !(f >= 0) || !std::isfinite(f)) return BSGPU_ERR_ARG;
    n_prod = (uint64_t)n_in * (uint64_t)(n_in + 1) / 2;
    long double c = (long double)n_freq * n_prod * n_time;
    if (c >= 4294967296.0L) return BSGPU_ERR_ARG;  // complex indices are 32-bit
    n_cplx = (uint64_t)n_freq * n_prod * (uint64_t)n_time;
    return BSGPU_OK;
}

VisParams vis_params(const WsLayout &L, void *ws, uint64_t n_in, uint64_t n_time, uint64_t n_prod,
                     double N, double f, int is_int = 0, const VisOpts &o = VisOpts(),
                     uint64_t n_freq = 0)
{
    VisParams v{};
    v.is_int = is_int;
    v.tslow = o.tslow;
    v.FP = (uint32_t)(n_freq * n_prod);
    v.qtab = L.qtab ? reinterpret_cast<const float *>((uint8_t *)ws + L.qtab) : nullptr;
    v.M = (uint32_t)(n_in * n_in);
    v.cft = L.cft ? reinterpret_cast<const float *>((uint8_t *)ws + L.cft) : nullptr;
    v.autos = reinterpret_cast<const float *>((uint8_t *)ws + L.autos);
    v.pairs = reinterpret_cast<const uint32_t *>((uint8_t *)ws + L.pairs);
    v.n_in = (uint32_t)n_in;
    v.T = (uint32_t)n_time;
    v.P = (uint32_t)n_prod;
    v.dT = fastdiv_init(v.T);
    v.dP = fastdiv_init(v.P);
    v.qT = (uint32_t)(32 / n_time);
    v.rT = (uint32_t)(32 % n_time);
    v.c = (float)(6.0 * f / N);   // q = 12 f s^2 with s^2 = A_i A_j / (2N)
    v.c2 = 2.0f * v.c;            // autos: s^2 = A_i^2 / N
    v.enabled = 1;
    return v;
}

// dtype and flags valid, and the full covariance only for small arrays
// (and not with the compensation, which corrects the diagonal approximation)
int vis_dtype_ok(int dtype, int flags, int64_t n_inputs = 1)
{
    if (dtype != BSGPU_VIS_F32 && dtype != BSGPU_VIS_I32) return 0;
    if (flags & ~(BSGPU_VIS_COMPENSATE | BSGPU_VIS_TIME_SLOWEST | BSGPU_VIS_FULL_COV)) return 0;
    if (flags & BSGPU_VIS_FULL_COV)
        return !(flags & BSGPU_VIS_COMPENSATE) && n_inputs <= (int64_t)FULL_MAX_INPUTS;
    return 1;
}

// The tables (autos, product indices) and, when asked, the compensated c
// per (freq, time) or the full-covariance q table: everything the rounding
// kernels read besides the cube.
int vis_prepare(const void *vis, const VisParams &v, int64_t n_freq, double N, double f,
                cudaStream_t s, double *s2 = nullptr)
{
    cudaError_t e = launch_vis_tables(reinterpret_cast<const float *>(vis), v, (uint32_t)n_freq, s);
    if (e != cudaSuccess) return BSGPU_ERR_CUDA;
    if (v.cft) e = launch_vis_compensation(vis, v, (uint32_t)n_freq, f, N, s);
    if (e == cudaSuccess && v.qtab)
        e = launch_full_noise(vis, v, (uint32_t)n_freq, f, N, s2, s);
    return e == cudaSuccess ? BSGPU_OK : BSGPU_ERR_CUDA;
}

}  // namespace

extern "C" {

const char *bsgpu_version(void) { return "bsgpu 0.1 (sm_103a)"; }

size_t bsgpu_compress_bound(size_t n_elem, size_t elem_size, size_t block_elems)
{
    Geometry g;
    if (geometry(n_elem, elem_size, block_elems, g) != BSGPU_OK) return 0;
    return (size_t)stream_bound(g);
}

size_t bsgpu_num_blocks(size_t n_elem, size_t elem_size, size_t block_elems)
{
    Geometry g;
    if (geometry(n_elem, elem_size, block_elems, g) != BSGPU_OK) return 0;
    return g.nb;
}

size_t bsgpu_workspace_size(int op, size_t n_elem, size_t elem_size, size_t block_elems)
{
    Geometry g{};
    if (op != BSGPU_OP_COMPRESS && op != BSGPU_OP_DECOMPRESS) return 0;
    if (geometry(n_elem, elem_size, block_elems, g) != BSGPU_OK) return 0;
    return ws_layout(op, g, 0, 0).total;
}

size_t bsgpu_vis_workspace_size_ex(int op, int64_t n_freq, int64_t n_inputs, int64_t n_time,
                                   size_t elem_size, size_t block_elems, int flags)
{
    uint64_t n_prod, n_cplx;
    if (op != BSGPU_OP_COMPRESS_VIS && op != BSGPU_OP_REDUCE_PRECISION) return 0;
    if (!vis_dtype_ok(BSGPU_VIS_F32, flags, n_inputs)) return 0;
    if (vis_check(n_freq, n_inputs, n_time, 1.0, 0.0, n_prod, n_cplx) != BSGPU_OK) return 0;
    Geometry g{};
    if (op == BSGPU_OP_COMPRESS_VIS) {
        if (elem_size != 4 && elem_size != 8) return 0;
        if (geometry(n_cplx * 8 / elem_size, elem_size, block_elems, g) != BSGPU_OK) return 0;
    }
    return ws_layout(op, g, (uint64_t)n_freq * n_inputs * n_time, n_prod, (uint64_t)n_time,
                     vis_opts(flags, n_freq, n_inputs, n_time))
        .total;
}

size_t bsgpu_vis_workspace_size(int op, int64_t n_freq, int64_t n_inputs, int64_t n_time,
                                size_t block_elems)
{
    return bsgpu_vis_workspace_size_ex(op, n_freq, n_inputs, n_time, 4, block_elems, 0);
}

int bsgpu_status(const void *ws, void *stream, int *status)
{
    if (!ws || !status) return BSGPU_ERR_ARG;
    int v = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&v, ws, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return BSGPU_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BSGPU_ERR_CUDA;
    *status = v;
    return BSGPU_OK;
}

int bsgpu_reduce_precision_ex(const void *in, void *out, int dtype, int64_t n_freq,
                              int64_t n_inputs, int64_t n_time, double N, double f, int flags,
                              void *ws, size_t ws_bytes, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_reduce_precision_ex");
    uint64_t n_prod, n_cplx;
    if (!vis_dtype_ok(dtype, flags, n_inputs)) return BSGPU_ERR_ARG;
    int rc = vis_check(n_freq, n_inputs, n_time, N, f, n_prod, n_cplx);
    if (rc) return rc;
    if (!in || !out || !ws) return BSGPU_ERR_ARG;
    if (!aligned16(in) || !aligned16(out) || !aligned16(ws)) return BSGPU_ERR_ALIGN;
    Geometry g{};
    uint64_t n_auto = (uint64_t)n_freq * n_inputs * n_time;
    const VisOpts o = vis_opts(flags, n_freq, n_inputs, n_time);
    WsLayout L = ws_layout(BSGPU_OP_REDUCE_PRECISION, g, n_auto, n_prod, 0, o);
    if (ws_bytes < L.total) return BSGPU_ERR_SPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws, 0, WS_HEADER, s) != cudaSuccess) return BSGPU_ERR_CUDA;
    VisParams v = vis_params(L, ws, n_inputs, n_time, n_prod, N, f, dtype == BSGPU_VIS_I32, o,
                             (uint64_t)n_freq);
    rc = vis_prepare(in, v, n_freq, N, f, s);
    if (rc) return rc;
    // 256-thread blocks, each warp rounding runs of 1024 samples
    uint64_t runs = (n_cplx + 1023) / 1024;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t want = (runs + 7) / 8, cap = (uint64_t)sms * 8;
    uint32_t grid = (uint32_t)(want < cap ? want : cap);
    if (grid == 0) grid = 1;
    return cuda_err(launch_reduce_precision(reinterpret_cast<const float *>(in),
                                            reinterpret_cast<float *>(out), n_cplx, v, grid, s));
}

int bsgpu_reduce_precision_c64(const void *in, void *out, int64_t n_freq, int64_t n_inputs,
                               int64_t n_time, double N, double f, void *ws, size_t ws_bytes,
                               void *stream)
{
    return bsgpu_reduce_precision_ex(in, out, BSGPU_VIS_F32, n_freq, n_inputs, n_time, N, f, 0,
                                     ws, ws_bytes, stream);
}

int bsgpu_full_noise_var(const void *vis, int dtype, int64_t n_freq, int64_t n_inputs,
                         int64_t n_time, double N, int flags, double *d_s2, void *ws,
                         size_t ws_bytes, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_full_noise_var");
    uint64_t n_prod, n_cplx;
    flags |= BSGPU_VIS_FULL_COV;
    if (!vis_dtype_ok(dtype, flags, n_inputs) || (flags & BSGPU_VIS_COMPENSATE))
        return BSGPU_ERR_ARG;
    int rc = vis_check(n_freq, n_inputs, n_time, N, 0.0, n_prod, n_cplx);
    if (rc) return rc;
    if (!vis || !d_s2 || !ws) return BSGPU_ERR_ARG;
    if (!aligned16(vis) || !aligned16(ws) || ((uintptr_t)d_s2 & 7u)) return BSGPU_ERR_ALIGN;
    Geometry g{};
    const VisOpts o = vis_opts(flags, n_freq, n_inputs, n_time);
    WsLayout L = ws_layout(BSGPU_OP_REDUCE_PRECISION, g, (uint64_t)n_freq * n_inputs * n_time,
                           n_prod, 0, o);
    if (ws_bytes < L.total) return BSGPU_ERR_SPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws, 0, WS_HEADER, s) != cudaSuccess) return BSGPU_ERR_CUDA;
    VisParams v = vis_params(L, ws, n_inputs, n_time, n_prod, N, 0.0, dtype == BSGPU_VIS_I32, o,
                             (uint64_t)n_freq);
    return vis_prepare(vis, v, n_freq, N, 0.0, s, d_s2);
}

int bsgpu_reorder_time(const void *in, void *out, uint64_t n_time, uint64_t n_series,
                       size_t elem_size, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_reorder_time");
    if (elem_size != 1 && elem_size != 2 && elem_size != 4 && elem_size != 8) return BSGPU_ERR_ARG;
    if (n_time == 0 || n_series == 0) return BSGPU_OK;
    if (!in || !out) return BSGPU_ERR_ARG;
    if (((uintptr_t)in | (uintptr_t)out) & (elem_size - 1)) return BSGPU_ERR_ALIGN;
    if (n_time > (1ull << 40) / n_series) return BSGPU_ERR_ARG;
    return cuda_err(launch_reorder_time(in, out, n_time, n_series, (uint32_t)elem_size,
                                        (cudaStream_t)stream));
}

static int shuffle_common(const void *in, void *out, size_t n_elem, size_t elem_size,
                          size_t block_elems, void *stream, bool inverse)
{
    Geometry g;
    int rc = geometry(n_elem, elem_size, block_elems, g);
    if (rc) return rc;
    if (n_elem == 0) return BSGPU_OK;
    if (!in || !out) return BSGPU_ERR_ARG;
    if (!aligned16(in) || !aligned16(out)) return BSGPU_ERR_ALIGN;
    CodecArgs a{};
    a.in = reinterpret_cast<const uint8_t *>(in);
    a.out = reinterpret_cast<uint8_t *>(out);
    a.n_elem = g.n;
    a.es = g.es;
    a.B = g.B;
    a.nb = g.nb;
    a.last_B = g.last_B;
    a.tail_elems = g.tail;
    uint32_t maxb = maxb_class(g.B * g.es);
    uint32_t grid = persistent_grid(shuffle_smem_bytes(maxb), g.nb ? g.nb : 1);
    return cuda_err(launch_shuffle(a, inverse, maxb, grid, (cudaStream_t)stream));
}

int bsgpu_bitshuffle(const void *in, void *out, size_t n_elem, size_t elem_size,
                     size_t block_elems, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_bitshuffle");
    return shuffle_common(in, out, n_elem, elem_size, block_elems, stream, false);
}

int bsgpu_bitunshuffle(const void *in, void *out, size_t n_elem, size_t elem_size,
                       size_t block_elems, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_bitunshuffle");
    return shuffle_common(in, out, n_elem, elem_size, block_elems, stream, true);
}

static int compress_common(const void *in, const Geometry &g, int level, void *out,
                           size_t out_cap, uint64_t *d_out_bytes, uint64_t *d_block_offsets,
                           void *ws, size_t ws_bytes, void *stream, const VisParams *vis,
                           const WsLayout &L)
{
    if (level < 0 || level > 1) return BSGPU_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (out_cap < stream_bound(g)) return BSGPU_ERR_SPACE;
    if (ws_bytes < L.total) return BSGPU_ERR_SPACE;
    CodecArgs a{};
    a.in = reinterpret_cast<const uint8_t *>(in);
    a.out = reinterpret_cast<uint8_t *>(out);
    a.out_cap = out_cap;
    a.out_bytes = d_out_bytes;
    a.block_offsets = d_block_offsets;
    a.status = reinterpret_cast<int *>(ws);
    a.tile_counter = reinterpret_cast<uint32_t *>((uint8_t *)ws + 4);
    a.tile_state = reinterpret_cast<uint64_t *>((uint8_t *)ws + L.state);
    a.n_elem = g.n;
    a.es = g.es;
    a.B = g.B;
    a.nb = g.nb;
    a.last_B = g.last_B;
    a.tail_elems = g.tail;
    a.level = level;
    if (vis) a.vis = *vis;
    if (cudaMemsetAsync(ws, 0, L.state + (size_t)g.nb * 8, s) != cudaSuccess)
        return BSGPU_ERR_CUDA;
    if (g.nb == 0) return cuda_err(launch_compress_small(a, s));
    // full blocks through the fast kernel when its slots are in the
    // workspace, the rest (a shortened last block, other shapes) through the
    // general one; both place blocks through the same look-back state
    const uint32_t nfull = g.nb - (g.last_B != g.B ? 1u : 0u);
    uint32_t done = 0;
    if (L.slots && nfull) {
        int dev = 0, sms = 148;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const bool ts = vis && vis->tslow;
        // 4-byte components of a cube whose time axis is not a multiple of 16
        const bool ps = vis && !vis->tslow && g.es == 4 && (vis->T % 16u) != 0;
        uint64_t grid = (uint64_t)sms * (ts ? compress_fast_tslow_blocks_per_sm(level, g.es)
                                            : ps ? compress_fast_ps_blocks_per_sm(level)
                                                 : compress_fast_blocks_per_sm(level, g.es));
        if (grid > nfull) grid = nfull;
        if (grid > FAST_MAX_WARPS) grid = FAST_MAX_WARPS;
        CodecArgs f = a;
        f.tile_begin = 0;
        f.tile_end = nfull;
        f.slots = reinterpret_cast<uint8_t *>(ws) + L.slots;
        f.nslot_warps = FAST_MAX_WARPS;
        f.tile_counter = reinterpret_cast<uint32_t *>((uint8_t *)ws + 4);
        cudaError_t e = ts   ? launch_compress_fast_tslow(f, (uint32_t)grid, s)
                        : ps ? launch_compress_fast_ps(f, (uint32_t)grid, s)
                             : launch_compress_fast(f, (uint32_t)grid, s);
        if (e != cudaSuccess) return BSGPU_ERR_CUDA;
        done = nfull;
    }
    if (done == g.nb) return BSGPU_OK;
    a.tile_begin = done;
    a.tile_end = g.nb;
    a.tile_counter = reinterpret_cast<uint32_t *>((uint8_t *)ws + 8);
    uint32_t maxb = maxb_class(g.B * g.es);
    a.slots = L.gslots ? reinterpret_cast<uint8_t *>(ws) + L.gslots : nullptr;
    a.nslot_warps = L.gslot_warps;
    uint32_t grid = persistent_grid(compress_smem_bytes(maxb, level, a.slots != nullptr), g.nb - done);
    if (a.slots && grid > a.nslot_warps) grid = a.nslot_warps;
    return cuda_err(launch_compress(a, maxb, grid, s));
}

int bsgpu_compress(const void *in, size_t n_elem, size_t elem_size, size_t block_elems,
                   int level, void *out, size_t out_cap, uint64_t *d_out_bytes, uint64_t *d_block_offsets,
                   void *ws, size_t ws_bytes, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_compress");
    Geometry g;
    int rc = geometry(n_elem, elem_size, block_elems, g);
    if (rc) return rc;
    if ((!in && n_elem) || !out || !d_out_bytes || !ws) return BSGPU_ERR_ARG;
    if ((in && !aligned16(in)) || !aligned16(ws) || ((uintptr_t)d_out_bytes & 7u) ||
        ((uintptr_t)d_block_offsets & 7u))
        return BSGPU_ERR_ALIGN;
    WsLayout L = ws_layout(BSGPU_OP_COMPRESS, g, 0, 0);
    return compress_common(in, g, level, out, out_cap, d_out_bytes, d_block_offsets, ws,
                           ws_bytes, stream, nullptr, L);
}

int bsgpu_compress_vis_ex(const void *vis, int dtype, int64_t n_freq, int64_t n_inputs,
                          int64_t n_time, double N, double f, int flags, size_t elem_size,
                          size_t block_elems, int level, void *out, size_t out_cap,
                          uint64_t *d_out_bytes, uint64_t *d_block_offsets, void *ws,
                          size_t ws_bytes, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_compress_vis_ex");
    uint64_t n_prod, n_cplx;
    if (!vis_dtype_ok(dtype, flags, n_inputs) || (elem_size != 4 && elem_size != 8))
        return BSGPU_ERR_ARG;
    int rc = vis_check(n_freq, n_inputs, n_time, N, f, n_prod, n_cplx);
    if (rc) return rc;
    Geometry g;
    rc = geometry(n_cplx * 8 / elem_size, elem_size, block_elems, g);
    if (rc) return rc;
    if (!vis || !out || !d_out_bytes || !ws) return BSGPU_ERR_ARG;
    if (!aligned16(vis) || !aligned16(ws) || ((uintptr_t)d_out_bytes & 7u) ||
        ((uintptr_t)d_block_offsets & 7u))
        return BSGPU_ERR_ALIGN;
    uint64_t n_auto = (uint64_t)n_freq * n_inputs * n_time;
    const VisOpts o = vis_opts(flags, n_freq, n_inputs, n_time);
    WsLayout L = ws_layout(BSGPU_OP_COMPRESS_VIS, g, n_auto, n_prod, (uint64_t)n_time, o);
    if (ws_bytes < L.total) return BSGPU_ERR_SPACE;
    if (level < 0 || level > 1) return BSGPU_ERR_ARG;
    if (out_cap < stream_bound(g)) return BSGPU_ERR_SPACE;
    VisParams v = vis_params(L, ws, n_inputs, n_time, n_prod, N, f, dtype == BSGPU_VIS_I32, o,
                             (uint64_t)n_freq);
    cudaStream_t s = (cudaStream_t)stream;
    rc = vis_prepare(vis, v, n_freq, N, f, s);
    if (rc) return rc;
    return compress_common(vis, g, level, out, out_cap, d_out_bytes, d_block_offsets, ws,
                           ws_bytes, stream, &v, L);
}

int bsgpu_compress_vis(const void *vis, int64_t n_freq, int64_t n_inputs, int64_t n_time,
                       double N, double f, size_t block_elems, int level, void *out,
                       size_t out_cap,
                       uint64_t *d_out_bytes, uint64_t *d_block_offsets, void *ws,
                       size_t ws_bytes, void *stream)
{
    return bsgpu_compress_vis_ex(vis, BSGPU_VIS_F32, n_freq, n_inputs, n_time, N, f, 0, 4,
                                 block_elems, level, out, out_cap, d_out_bytes, d_block_offsets,
                                 ws, ws_bytes, stream);
}

int bsgpu_decompress(const void *in, size_t in_bytes, void *out, size_t n_elem, size_t elem_size,
                     size_t block_elems, const uint64_t *d_block_offsets, void *ws,
                     size_t ws_bytes, void *stream)
{
    const NvtxRange nvtx_range("bsgpu_decompress");
    Geometry g;
    int rc = geometry(n_elem, elem_size, block_elems, g);
    if (rc) return rc;
    if (!in || (!out && n_elem) || !ws) return BSGPU_ERR_ARG;
    if ((out && !aligned16(out)) || !aligned16(ws) || ((uintptr_t)d_block_offsets & 7u))
        return BSGPU_ERR_ALIGN;
    WsLayout L = ws_layout(BSGPU_OP_DECOMPRESS, g, 0, 0);
    if (ws_bytes < L.total) return BSGPU_ERR_SPACE;
    cudaStream_t s = (cudaStream_t)stream;
    CodecArgs a{};
    a.in = reinterpret_cast<const uint8_t *>(in);
    a.out = reinterpret_cast<uint8_t *>(out);
    a.in_bytes = in_bytes;
    a.status = reinterpret_cast<int *>(ws);
    a.tile_counter = reinterpret_cast<uint32_t *>((uint8_t *)ws + 4);
    a.n_elem = g.n;
    a.es = g.es;
    a.B = g.B;
    a.nb = g.nb;
    a.last_B = g.last_B;
    a.tail_elems = g.tail;
    if (cudaMemsetAsync(ws, 0, WS_HEADER, s) != cudaSuccess) return BSGPU_ERR_CUDA;
    if (d_block_offsets) {
        a.block_offsets = const_cast<uint64_t *>(d_block_offsets);
    } else if (g.nb) {
        a.block_offsets = reinterpret_cast<uint64_t *>((uint8_t *)ws + L.offsets);
        cudaError_t e = launch_chain_walk(a, a.block_offsets, (uint8_t *)ws + L.segs, s);
        if (e != cudaSuccess) return BSGPU_ERR_CUDA;
    }
    uint32_t maxb = maxb_class(g.B * g.es);
    if (g.nb && !(maxb <= 8192 && g.es != 1) && (g.B * g.es) % 16u == 0) {
        // blocks over 8 KiB and 1-byte elements: decoded in place as well
        const uint32_t grid = persistent_grid(decompress_inplace_any_smem_bytes(maxb), g.nb);
        return cuda_err(launch_decompress_inplace_any(a, maxb, grid, s));
    }
    uint32_t grid = persistent_grid(decompress_smem_bytes(maxb), g.nb ? g.nb : 1);
    if (maxb <= 8192 && (g.es == 2 || g.es == 4 || g.es == 8)) {
        // the in-place kernel: as many warps as fit, never more than the blocks
        int dev = 0, sms = 148;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const uint64_t want = (uint64_t)sms * decompress_inplace_blocks_per_sm(g.es);
        grid = (uint32_t)(want < g.nb ? want : (g.nb ? g.nb : 1));
    }
    return cuda_err(launch_decompress(a, maxb, grid, s));
}

}  // extern "C"
