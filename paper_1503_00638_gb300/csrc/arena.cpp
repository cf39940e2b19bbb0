// Offset allocator for a fixed device arena (host code only).
//
// The serving layer keeps one device allocation of a fixed capacity (the
// admission cap) and hands out byte ranges of it to requests as they are
// admitted; a request whose ranges do not fit waits.  This file manages the
// offsets: best fit over a size-ordered index of free ranges, neighbours
// merged on free, every range aligned.  It never touches device memory.
#include <cstdint>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <unordered_map>

#include "../../include/bsgpu.h"

namespace {

struct Arena {
    uint64_t cap = 0, align = 256;
    std::map<uint64_t, uint64_t> free_by_off;            // offset -> size
    std::multimap<uint64_t, uint64_t> free_by_size;      // size -> offset
    std::unordered_map<uint64_t, uint64_t> used;         // offset -> size
    uint64_t used_bytes = 0, high_water = 0;
    std::mutex m;

    void insert_free(uint64_t off, uint64_t size)
    {
        free_by_off.emplace(off, size);
        free_by_size.emplace(size, off);
    }

    void erase_free(std::map<uint64_t, uint64_t>::iterator it)
    {
        auto range = free_by_size.equal_range(it->second);
        for (auto s = range.first; s != range.second; ++s) {
            if (s->second == it->first) {
                free_by_size.erase(s);
                break;
            }
        }
        free_by_off.erase(it);
    }
};

}  // namespace

extern "C" {

void *bsgpu_arena_create(uint64_t capacity, uint64_t align)
{
    if (capacity == 0 || align == 0 || (align & (align - 1))) return nullptr;
    Arena *a = new (std::nothrow) Arena;
    if (!a) return nullptr;
    a->align = align;
    a->cap = capacity / align * align;
    if (a->cap) a->insert_free(0, a->cap);
    return a;
}

void bsgpu_arena_destroy(void *arena) { delete static_cast<Arena *>(arena); }

int bsgpu_arena_alloc(void *arena, uint64_t bytes, uint64_t *offset)
{
    Arena *a = static_cast<Arena *>(arena);
    if (!a || !offset) return BSGPU_ERR_ARG;
    const uint64_t need = (bytes ? bytes : 1) + a->align - 1;
    if (need < bytes) return BSGPU_ERR_SPACE;  // overflow
    const uint64_t size = need / a->align * a->align;
    std::lock_guard<std::mutex> g(a->m);
    auto s = a->free_by_size.lower_bound(size);  // best fit: smallest range that fits
    if (s == a->free_by_size.end()) return BSGPU_ERR_SPACE;
    const uint64_t off = s->second, have = s->first;
    a->erase_free(a->free_by_off.find(off));
    if (have > size) a->insert_free(off + size, have - size);
    a->used.emplace(off, size);
    a->used_bytes += size;
    if (a->used_bytes > a->high_water) a->high_water = a->used_bytes;
    *offset = off;
    return BSGPU_OK;
}

int bsgpu_arena_free(void *arena, uint64_t offset)
{
    Arena *a = static_cast<Arena *>(arena);
    if (!a) return BSGPU_ERR_ARG;
    std::lock_guard<std::mutex> g(a->m);
    auto u = a->used.find(offset);
    if (u == a->used.end()) return BSGPU_ERR_ARG;
    uint64_t off = u->first, size = u->second;
    a->used.erase(u);
    a->used_bytes -= size;
    // merge with the free neighbours on both sides
    auto next = a->free_by_off.lower_bound(off);
    if (next != a->free_by_off.end() && next->first == off + size) {
        size += next->second;
        a->erase_free(next);
    }
    auto after = a->free_by_off.lower_bound(off);
    if (after != a->free_by_off.begin()) {
        auto prev = std::prev(after);
        if (prev->first + prev->second == off) {
            off = prev->first;
            size += prev->second;
            a->erase_free(prev);
        }
    }
    a->insert_free(off, size);
    return BSGPU_OK;
}

int bsgpu_arena_stats(const void *arena, uint64_t *used_bytes, uint64_t *largest_free,
                      uint64_t *high_water, uint64_t *n_free_ranges)
{
    const Arena *a = static_cast<const Arena *>(arena);
    if (!a) return BSGPU_ERR_ARG;
    std::lock_guard<std::mutex> g(const_cast<Arena *>(a)->m);
    if (used_bytes) *used_bytes = a->used_bytes;
    if (largest_free) *largest_free = a->free_by_size.empty() ? 0 : a->free_by_size.rbegin()->first;
    if (high_water) *high_water = a->high_water;
    if (n_free_ranges) *n_free_ranges = a->free_by_off.size();
    return BSGPU_OK;
}

}  // extern "C"
