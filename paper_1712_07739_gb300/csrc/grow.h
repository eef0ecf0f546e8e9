// Capacity-tracked buffer sets (host code; no CUDA dependency, so the CPU
// tests compile it with a fake allocator).
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <initializer_list>

struct GrowBuf {
    void **ptr;    // where the buffer's pointer lives
    size_t bytes;  // size it must have for the requested capacity
};

// Make every buffer of a set hold `need` units, reallocating the whole set
// when `need` exceeds `cap`.  The capacity is cleared before the old buffers
// are released and recorded only after every allocation of the set has
// succeeded; when one fails, the buffers already allocated are released
// again, so a failed call leaves the set empty (null pointers, capacity 0)
// and the next call allocates afresh instead of trusting a stale capacity.
// alloc(void **, size_t) returns 0 on success; release(void *) frees.
// Returns 0, or -1 when an allocation failed.
template <typename Alloc, typename Release>
int grow_set(int64_t &cap, int64_t need, const GrowBuf *bufs, int n, Alloc alloc, Release release) {
    if (need <= cap) return 0;
    cap = 0;
    for (int i = 0; i < n; ++i) {
        if (*bufs[i].ptr) release(*bufs[i].ptr);
        *bufs[i].ptr = nullptr;
    }
    for (int i = 0; i < n; ++i)
        if (alloc(bufs[i].ptr, bufs[i].bytes) != 0) {
            for (int j = 0; j < n; ++j) {
                if (j < i && *bufs[j].ptr) release(*bufs[j].ptr);
                *bufs[j].ptr = nullptr;
            }
            return -1;
        }
    cap = need;
    return 0;
}

template <typename Alloc, typename Release>
int grow_set(int64_t &cap, int64_t need, std::initializer_list<GrowBuf> bufs, Alloc alloc, Release release) {
    return grow_set(cap, need, bufs.begin(), int(bufs.size()), alloc, release);
}
