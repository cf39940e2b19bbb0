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

// Held by every device that loads the library, for the life of the process.
static __device__ __align__(256) uint8_t g_compress_scratch[NOALLOC_BYTES];

// A device-side failure (a bounded wait that ran out) turns the reported
// stream length into 0; a valid stream is at least 12 bytes long.
__global__ void noalloc_report_kernel(const int *status, uint64_t *out_bytes)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && *status != 0) *out_bytes = 0;
}

constexpr int MAX_DEVICES = 64;
std::once_flag g_once[MAX_DEVICES];
void *g_scratch_ptr[MAX_DEVICES];
cudaError_t g_scratch_err[MAX_DEVICES];

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device, with that device current.
int scratch_on_current_device(void **ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BSGPU_ERR_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return BSGPU_ERR_ARG;
    std::call_once(g_once[dev], [dev] {
        g_scratch_err[dev] = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_compress_scratch);
    });
    if (g_scratch_err[dev] != cudaSuccess) return BSGPU_ERR_CUDA;
    *ptr = g_scratch_ptr[dev];
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
    int rc = scratch_on_current_device(&scratch);
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
    noalloc_report_kernel<<<1, 32, 0, s>>>(a.status, d_out_bytes);
    return cudaGetLastError() == cudaSuccess ? BSGPU_OK : BSGPU_ERR_CUDA;
}
