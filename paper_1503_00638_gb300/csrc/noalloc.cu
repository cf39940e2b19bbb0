// bsgpu_compress_noalloc: bsgpu_compress without a caller-provided workspace.
//
// Some callers are handed buffers but may not allocate device memory: a
// filter callback of an I/O library receives only the chunk's input and
// output buffers; a real-time acquisition loop allocates everything at start
// and must not call cudaMalloc afterwards (it synchronizes the device and can
// stall the loop); a process whose device memory is wholly owned by a pool.
// For them this entry point keeps its scratch (the status word, the tile
// counter and the per-block look-back state of the compress kernel) in a
// fixed array in device memory that belongs to the library.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/bsgpu.h"
#include "kernels.cuh"

using namespace bsg;

namespace {

constexpr uint32_t NOALLOC_MAX_BLOCKS = 131072;   // 1 GiB of input at 8 KiB blocks
constexpr size_t NOALLOC_HEADER = 256;            // status word, tile counter
constexpr size_t NOALLOC_BYTES = NOALLOC_HEADER + 8ull * NOALLOC_MAX_BLOCKS;

// One copy in every context the module is loaded into, for the life of the
// process (with lazy module loading, from the first call in that context).
static __device__ __align__(256) uint8_t g_compress_scratch[NOALLOC_BYTES];

// Any device-side failure recorded in the status word (a bounded wait that
// ran out, or any other error code) turns the reported stream length into
// 0; a valid stream is at least 12 bytes long.
__global__ void noalloc_report_kernel(const int *status, uint64_t *out_bytes)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && *status != 0) *out_bytes = 0;
}

// Device address of the scratch array in the calling thread's current
// context.  In host code the array's name is only a host-side stand-in; its
// device address belongs to a context (the module is loaded per context), so
// the lookup is cached per context, keyed by the driver's context id (ids
// are never reused, so a context created after cudaDeviceReset, or a second
// context on the same device, gets its own lookup).  Failures are not
// cached.  The driver's context queries are reached through the runtime's
// entry-point lookup, so the library does not link the driver library.
typedef int (*CtxGetCurrentFn)(CUcontext *);
typedef int (*CtxGetIdFn)(CUcontext, unsigned long long *);

constexpr int CACHE_SLOTS = 64;
struct ScratchSlot {
    unsigned long long ctx_id;
    void *ptr;
};
std::mutex g_mu;
ScratchSlot g_slots[CACHE_SLOTS];
int g_nslots = 0;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_fns_tried = false;

// Id of the current context, or false when it cannot be had (no driver
// entry points, or no context current yet).
bool current_context_id(unsigned long long *id)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_fns_tried) {
            g_fns_tried = true;
            void *f1 = nullptr, *f2 = nullptr;
            cudaDriverEntryPointQueryResult q1, q2;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                                 &q1) == cudaSuccess &&
                q1 == cudaDriverEntryPointSuccess &&
                cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault,
                                                 &q2) == cudaSuccess &&
                q2 == cudaDriverEntryPointSuccess) {
                g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
                g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
            }
        }
    }
    if (!g_ctx_current || !g_ctx_id) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != 0 || ctx == nullptr) return false;
    return g_ctx_id(ctx, id) == 0;
}

int scratch_in_current_context(void **ptr)
{
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    if (have_id) {
        std::lock_guard<std::mutex> lk(g_mu);
        for (int k = 0; k < g_nslots; k++)
            if (g_slots[k].ctx_id == id) {
                *ptr = g_slots[k].ptr;
                return BSGPU_OK;
            }
    }
    // first call in this context: the lookup loads the library's module into
    // the context (and, with no context current yet, makes the device's
    // primary context current)
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_compress_scratch) != cudaSuccess || p == nullptr)
        return BSGPU_ERR_CUDA;
    if (!have_id) have_id = current_context_id(&id);
    if (have_id) {
        std::lock_guard<std::mutex> lk(g_mu);
        bool known = false;
        for (int k = 0; k < g_nslots; k++) known = known || g_slots[k].ctx_id == id;
        if (!known && g_nslots < CACHE_SLOTS) g_slots[g_nslots++] = ScratchSlot{id, p};
    }
    *ptr = p;
    return BSGPU_OK;
}

}  // namespace

extern "C" int bsgpu_compress_noalloc(const void *in, size_t n_elem, size_t elem_size,
                                      size_t block_elems, int level, void *out, size_t out_cap,
                                      uint64_t *d_out_bytes, uint64_t *d_block_offsets,
                                      void *stream)
{
    const size_t bound = bsgpu_compress_bound(n_elem, elem_size, block_elems);
    if (bound == 0 || level < 0 || level > 1) return BSGPU_ERR_ARG;
    if ((!in && n_elem) || !out || !d_out_bytes) return BSGPU_ERR_ARG;
    if ((in && ((uintptr_t)in & 15u)) || ((uintptr_t)d_out_bytes & 7u) ||
        ((uintptr_t)d_block_offsets & 7u))
        return BSGPU_ERR_ALIGN;
    if (out_cap < bound) return BSGPU_ERR_SPACE;
    const size_t nb = bsgpu_num_blocks(n_elem, elem_size, block_elems);
    if (nb > NOALLOC_MAX_BLOCKS) return BSGPU_ERR_SPACE;  // beyond the fixed scratch

    void *scratch = nullptr;
    int rc = scratch_in_current_context(&scratch);
    if (rc != BSGPU_OK) return rc;

    const uint32_t B = (uint32_t)(block_elems ? block_elems : 4096 / elem_size);
    const uint64_t rem = n_elem % B, last = rem - rem % 8;
    CodecArgs a{};
    a.in = reinterpret_cast<const uint8_t *>(in);
    a.out = reinterpret_cast<uint8_t *>(out);
    a.out_cap = out_cap;
    a.out_bytes = d_out_bytes;
    a.block_offsets = d_block_offsets;
    a.status = reinterpret_cast<int *>(scratch);
    a.tile_counter = reinterpret_cast<uint32_t *>((uint8_t *)scratch + 4);
    a.tile_state = reinterpret_cast<uint64_t *>((uint8_t *)scratch + NOALLOC_HEADER);
    a.n_elem = n_elem;
    a.es = (uint32_t)elem_size;
    a.B = B;
    a.nb = (uint32_t)nb;
    a.last_B = (uint32_t)(last ? last : B);
    a.tail_elems = (uint32_t)(rem % 8);
    a.level = level;
    a.tile_begin = 0;
    a.tile_end = (uint32_t)nb;

    // the array keeps the previous call's contents: clear what starts at zero
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(scratch, 0, NOALLOC_HEADER + 8 * nb, s) != cudaSuccess)
        return BSGPU_ERR_CUDA;
    cudaError_t e;
    if (nb == 0) {
        e = launch_compress_small(a, s);
    } else {
        const uint32_t maxb = maxb_class(B * (uint32_t)elem_size);
        int dev = 0, sms = 148, smem_sm = 228 * 1024;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        uint32_t per_sm = (uint32_t)(smem_sm / (compress_smem_bytes(maxb, level) + 1024));
        per_sm = per_sm == 0 ? 1 : (per_sm > 32 ? 32 : per_sm);
        uint64_t grid = (uint64_t)sms * per_sm;
        if (grid > nb) grid = nb;
        e = launch_compress(a, maxb, (uint32_t)grid, s);
    }
    if (e != cudaSuccess) return BSGPU_ERR_CUDA;
    // launched through cudaLaunchKernel, whose return value is this launch's
    // own error (an error left by an unrelated earlier launch is not taken
    // for it)
    const int *st = a.status;
    void *args[] = {(void *)&st, (void *)&d_out_bytes};
    e = cudaLaunchKernel((const void *)noalloc_report_kernel, dim3(1), dim3(32), args, 0, s);
    return e == cudaSuccess ? BSGPU_OK : BSGPU_ERR_CUDA;
}
