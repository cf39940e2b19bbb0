// Host emulation of one CUDA warp for CPU tests of warp-level device code:
// 32 std::threads run the same function; every warp collective (ballot,
// shuffle, match, syncwarp) is a barrier at which the lanes exchange values.
#pragma once
#include <barrier>
#include <thread>
#include <mutex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <cstdio>
#include <cstdlib>
#include <vector_types.h>      // uint4 and friends; defines __host__ / __device__ as no-ops
#include <vector_functions.h>
#define BSG_WARP_EMU 1
struct EmuTid { unsigned x; };
inline thread_local EmuTid threadIdx;
struct WarpCtx { std::barrier<> bar{32}; uint32_t v[32]; uint64_t v64[32]; std::mutex mu; };
inline WarpCtx* g_warp;
inline void __syncwarp(unsigned = 0xffffffffu) { g_warp->bar.arrive_and_wait(); }
inline uint32_t __ballot_sync(uint32_t, int p) { g_warp->v[threadIdx.x] = p ? 1 : 0; g_warp->bar.arrive_and_wait(); uint32_t r = 0; for (int i = 0; i < 32; i++) r |= g_warp->v[i] << i; g_warp->bar.arrive_and_wait(); return r; }
template <class T> inline T __shfl_sync(uint32_t, T x, int src) { static_assert(sizeof(T)==4); uint32_t u; memcpy(&u,&x,4); g_warp->v[threadIdx.x] = u; g_warp->bar.arrive_and_wait(); uint32_t r = g_warp->v[src & 31]; g_warp->bar.arrive_and_wait(); T o; memcpy(&o,&r,4); return o; }
template <class T> inline T __shfl_up_sync(uint32_t, T x, unsigned d) { static_assert(sizeof(T)==4); uint32_t u; memcpy(&u,&x,4); g_warp->v[threadIdx.x] = u; g_warp->bar.arrive_and_wait(); uint32_t r = threadIdx.x >= d ? g_warp->v[threadIdx.x - d] : u; g_warp->bar.arrive_and_wait(); T o; memcpy(&o,&r,4); return o; }
template <class T> inline T __shfl_down_sync(uint32_t, T x, unsigned d) { static_assert(sizeof(T)==4); uint32_t u; memcpy(&u,&x,4); g_warp->v[threadIdx.x] = u; g_warp->bar.arrive_and_wait(); uint32_t r = threadIdx.x + d < 32 ? g_warp->v[threadIdx.x + d] : u; g_warp->bar.arrive_and_wait(); T o; memcpy(&o,&r,4); return o; }
template <class T> inline T __shfl_xor_sync(uint32_t, T x, int m) { uint64_t u = 0; memcpy(&u,&x,sizeof(T)); static thread_local int dummy; (void)dummy; uint64_t *v64 = reinterpret_cast<uint64_t *>(g_warp->v64); v64[threadIdx.x] = u; g_warp->bar.arrive_and_wait(); uint64_t r = v64[threadIdx.x ^ m]; g_warp->bar.arrive_and_wait(); T o; memcpy(&o,&r,sizeof(T)); return o; }
inline uint32_t __match_any_sync(uint32_t, uint32_t x) { g_warp->v[threadIdx.x] = x; g_warp->bar.arrive_and_wait(); uint32_t r = 0; for (int i = 0; i < 32; i++) if (g_warp->v[i] == x) r |= 1u << i; g_warp->bar.arrive_and_wait(); return r; }
inline int __ffs(uint32_t x) { return x ? __builtin_ctz(x) + 1 : 0; }
inline int __popc(uint32_t x) { return __builtin_popcount(x); }
inline int __clz(uint32_t x) { return x ? __builtin_clz(x) : 32; }
inline uint32_t atomicMax(uint32_t* p, uint32_t v) { std::lock_guard<std::mutex> g(g_warp->mu); uint32_t o = *p; if (v > o) *p = v; return o; }
inline void __nanosleep(unsigned) {}
inline void emu_check_aligned4(const void *p)
{
    if ((uintptr_t)p & 3u) {
        fprintf(stderr, "misaligned 4-byte access base %p\n", p);
        abort();
    }
}
namespace bsg { inline uint32_t lanemask_lt() { return (1u << threadIdx.x) - 1u; } }
inline void run_warp(const std::function<void()>& f) {
  WarpCtx ctx; g_warp = &ctx; std::thread t[32];
  for (int i = 0; i < 32; i++) t[i] = std::thread([&, i] { threadIdx.x = i; f(); });
  for (auto& x : t) x.join();
}
