// arena.h -- first-fit allocator with coalescing over an address range.
// Pure host bookkeeping: it never touches the memory it manages.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <map>
#include <string>
#include <unordered_map>

namespace rearr {

class Arena {
public:
    static constexpr size_t kAlign = 256;

    Arena(uintptr_t base, size_t bytes);

    // First free block (lowest address) that fits; false if none does.
    bool alloc(size_t bytes, uintptr_t &addr);
    // False if addr is not the start of a live block.
    bool free(uintptr_t addr);

    size_t used() const { return used_; }
    size_t capacity() const { return size_; }
    size_t largest_free() const;
    size_t n_blocks() const { return live_.size(); }
    static size_t round(size_t bytes) { return bytes == 0 ? kAlign : (bytes + kAlign - 1) / kAlign * kAlign; }

private:
    uintptr_t base_;
    size_t size_;
    size_t used_ = 0;
    std::map<uintptr_t, size_t> free_;            // start -> size, disjoint, coalesced
    std::unordered_map<uintptr_t, size_t> live_;  // start -> size
};

}  // namespace rearr
