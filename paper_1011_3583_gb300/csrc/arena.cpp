// arena.cpp -- first-fit allocator of the serving slab, and its C ABI.
#include "arena.h"

#include <new>

#include "../../include/librearr_serve.h"

namespace rearr {

rearr_status fail(rearr_status st, const std::string &msg);

Arena::Arena(uintptr_t base, size_t bytes)
{
    // Work on 256-byte boundaries inside [base, base + bytes).
    const uintptr_t b = (base + kAlign - 1) / kAlign * kAlign;
    const uintptr_t e = (base + bytes) / kAlign * kAlign;
    base_ = b;
    size_ = e > b ? size_t(e - b) : 0;
    if (size_) free_[base_] = size_;
}

bool Arena::alloc(size_t bytes, uintptr_t &addr)
{
    const size_t need = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
        if (it->second < need) continue;
        addr = it->first;
        const size_t rest = it->second - need;
        free_.erase(it);
        if (rest) free_[addr + need] = rest;
        live_[addr] = need;
        used_ += need;
        return true;
    }
    return false;
}

bool Arena::free(uintptr_t addr)
{
    auto lv = live_.find(addr);
    if (lv == live_.end()) return false;
    size_t size = lv->second;
    live_.erase(lv);
    used_ -= size;
    uintptr_t start = addr;
    auto next = free_.lower_bound(addr);
    if (next != free_.end() && next->first == addr + size) {  // merge with the following block
        size += next->second;
        next = free_.erase(next);
    }
    if (next != free_.begin()) {  // merge with the preceding block
        auto prev = std::prev(next);
        if (prev->first + prev->second == start) {
            start = prev->first;
            size += prev->second;
            free_.erase(prev);
        }
    }
    free_[start] = size;
    return true;
}

size_t Arena::largest_free() const
{
    size_t m = 0;
    for (auto &kv : free_) m = kv.second > m ? kv.second : m;
    return m;
}

}  // namespace rearr

struct rearr_arena {
    rearr::Arena a;
    rearr_arena(uintptr_t b, size_t n) : a(b, n) {}
};

using rearr::fail;

extern "C" {

rearr_status rearr_arena_create(uintptr_t base, size_t bytes, rearr_arena **arena)
{
    if (!arena) return fail(REARR_EINVAL, "rearr_arena_create: arena is NULL");
    if (base == 0 || bytes < rearr::Arena::kAlign) return fail(REARR_EINVAL, "rearr_arena_create: empty range");
    *arena = new (std::nothrow) rearr_arena(base, bytes);
    return *arena ? REARR_OK : fail(REARR_ENOMEM, "rearr_arena_create: out of host memory");
}

rearr_status rearr_arena_alloc(rearr_arena *arena, size_t bytes, uintptr_t *addr)
{
    if (!arena || !addr) return fail(REARR_EINVAL, "rearr_arena_alloc: NULL argument");
    if (!arena->a.alloc(bytes, *addr)) return fail(REARR_ENOMEM, "rearr_arena_alloc: no free block fits");
    return REARR_OK;
}

rearr_status rearr_arena_free(rearr_arena *arena, uintptr_t addr)
{
    if (!arena) return fail(REARR_EINVAL, "rearr_arena_free: arena is NULL");
    if (!arena->a.free(addr)) return fail(REARR_EINVAL, "rearr_arena_free: not a live block");
    return REARR_OK;
}

rearr_status rearr_arena_stats(const rearr_arena *arena, size_t *used, size_t *free_bytes, size_t *largest_free,
                               size_t *n_blocks)
{
    if (!arena) return fail(REARR_EINVAL, "rearr_arena_stats: arena is NULL");
    if (used) *used = arena->a.used();
    if (free_bytes) *free_bytes = arena->a.capacity() - arena->a.used();
    if (largest_free) *largest_free = arena->a.largest_free();
    if (n_blocks) *n_blocks = arena->a.n_blocks();
    return REARR_OK;
}

void rearr_arena_destroy(rearr_arena *arena) { delete arena; }

}  // extern "C"
