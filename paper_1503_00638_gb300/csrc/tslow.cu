// The fast compress kernel for time-slowest cubes ([T][F P] samples, the
// instrument's order before the post-acquisition reorder of Sec. 2): each
// full block is gathered into time-fastest order in shared memory and then
// rounded, shuffled and coded exactly like a block of a time-fastest cube;
// time-slowest cubes whose time axis is not a multiple of 16 are gathered and
// rounded sample by sample; and so are time-fastest cubes of 4-byte
// components with such a time axis (rounded sample by sample, then shuffled).  Kept in their
// own translation unit so the in-order kernels compile without these paths
// and the build compiles both in parallel.
#include <cuda_runtime.h>

#include "compress_fast.cuh"

namespace bsg {

uint32_t compress_fast_tslow_blocks_per_sm(int level, uint32_t es)
{
    int n = 0;
    const uint32_t smem = compress_fast_smem_bytes(level);
    cudaError_t e;
    if (es == 8)
        e = level >= 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, compress_fast_kernel<1, 8, false, true>, 32, smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, compress_fast_kernel<0, 8, false, true>, 32, smem);
    else
        e = level >= 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, compress_fast_kernel<1, 4, false, true>, 32, smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &n, compress_fast_kernel<0, 4, false, true>, 32, smem);
    return e == cudaSuccess && n > 0 ? (uint32_t)n : 1u;
}

cudaError_t launch_compress_fast_tslow(const CodecArgs &a, uint32_t grid, cudaStream_t s)
{
    const uint32_t smem = compress_fast_smem_bytes(a.level);
    // series of 16 samples only when they cannot straddle products and fill
    // whole blocks; otherwise samples are gathered and rounded one by one
    // (the same occupancy: the same registers and shared memory)
    if (a.vis.T % 16u != 0 || ((uint64_t)a.B * a.es) % 128u != 0) {
        if (a.es == 8)
            return a.level >= 1
                       ? launch_warp_kernel(compress_fast_kernel<1, 8, false, true, true>, smem,
                                            grid, s, a)
                       : launch_warp_kernel(compress_fast_kernel<0, 8, false, true, true>, smem,
                                            grid, s, a);
        return a.level >= 1
                   ? launch_warp_kernel(compress_fast_kernel<1, 4, false, true, true>, smem, grid,
                                        s, a)
                   : launch_warp_kernel(compress_fast_kernel<0, 4, false, true, true>, smem, grid,
                                        s, a);
    }
    if (a.es == 8)
        return a.level >= 1
                   ? launch_warp_kernel(compress_fast_kernel<1, 8, false, true>, smem, grid, s, a)
                   : launch_warp_kernel(compress_fast_kernel<0, 8, false, true>, smem, grid, s, a);
    if (a.vis.is_int || a.vis.cft || a.vis.qtab)
        return a.level >= 1
                   ? launch_warp_kernel(compress_fast_kernel<1, 4, true, true>, smem, grid, s, a)
                   : launch_warp_kernel(compress_fast_kernel<0, 4, true, true>, smem, grid, s, a);
    return a.level >= 1
               ? launch_warp_kernel(compress_fast_kernel<1, 4, false, true>, smem, grid, s, a)
               : launch_warp_kernel(compress_fast_kernel<0, 4, false, true>, smem, grid, s, a);
}

// Cubes of 4-byte components whose time axis is not a multiple of 16: the
// fast kernel rounding each sample before the transpose (PS).
uint32_t compress_fast_ps_blocks_per_sm(int level)
{
    int n = 0;
    const uint32_t smem = compress_fast_smem_bytes(level);
    const cudaError_t e =
        level >= 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                         &n, compress_fast_kernel<1, 4, false, false, true>, 32, smem)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                         &n, compress_fast_kernel<0, 4, false, false, true>, 32, smem);
    return e == cudaSuccess && n > 0 ? (uint32_t)n : 1u;
}

cudaError_t launch_compress_fast_ps(const CodecArgs &a, uint32_t grid, cudaStream_t s)
{
    const uint32_t smem = compress_fast_smem_bytes(a.level);
    return a.level >= 1
               ? launch_warp_kernel(compress_fast_kernel<1, 4, false, false, true>, smem, grid, s, a)
               : launch_warp_kernel(compress_fast_kernel<0, 4, false, false, true>, smem, grid, s, a);
}

}  // namespace bsg
