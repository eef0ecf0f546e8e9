// Host check of grow_set (paper_1712_07739_gb300/csrc/grow.h) with a fake
// allocator that fails on request: a failed growth must leave the set empty
// (null pointers, capacity 0, nothing leaked) so the next call allocates again.
#include <cstdio>
#include <cstdlib>
#include <set>

#include "../paper_1712_07739_gb300/csrc/grow.h"

static std::set<void *> live;
static int fail_at = -1, calls = 0;

static int fake_alloc(void **p, size_t n) {
    if (calls++ == fail_at) return -1;
    *p = std::malloc(n ? n : 1);
    live.insert(*p);
    return 0;
}
static void fake_free(void *p) {
    if (!live.erase(p)) {
        std::printf("FAIL: free of a pointer that is not live\n");
        std::exit(1);
    }
    std::free(p);
}

#define CHECK(c)                                              \
    do {                                                      \
        if (!(c)) {                                           \
            std::printf("FAIL line %d: %s\n", __LINE__, #c); \
            return 1;                                         \
        }                                                     \
    } while (0)

int main() {
    void *a = nullptr, *b = nullptr, *c = nullptr;
    int64_t cap = 0;
    // first growth
    CHECK(grow_set(cap, 10, {{&a, 10}, {&b, 20}, {&c, 30}}, fake_alloc, fake_free) == 0);
    CHECK(cap == 10 && a && b && c && live.size() == 3);
    // within capacity: nothing happens
    calls = 0;
    CHECK(grow_set(cap, 8, {{&a, 8}, {&b, 16}, {&c, 24}}, fake_alloc, fake_free) == 0);
    CHECK(calls == 0 && cap == 10 && live.size() == 3);
    // growth whose second allocation fails: set empty, capacity 0, no leak
    calls = 0;
    fail_at = 1;
    CHECK(grow_set(cap, 100, {{&a, 100}, {&b, 200}, {&c, 300}}, fake_alloc, fake_free) == -1);
    CHECK(cap == 0 && !a && !b && !c && live.empty());
    // the next call, even for a size below the old capacity, allocates afresh
    calls = 0;
    fail_at = -1;
    CHECK(grow_set(cap, 5, {{&a, 5}, {&b, 10}, {&c, 15}}, fake_alloc, fake_free) == 0);
    CHECK(calls == 3 && cap == 5 && a && b && c && live.size() == 3);
    // failure of the first allocation of a set
    calls = 0;
    fail_at = 0;
    CHECK(grow_set(cap, 50, {{&a, 50}, {&b, 50}, {&c, 50}}, fake_alloc, fake_free) == -1);
    CHECK(cap == 0 && !a && !b && !c && live.empty());
    std::printf("OK\n");
    return 0;
}
