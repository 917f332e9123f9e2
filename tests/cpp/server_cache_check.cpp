// Checks of the solve server's factor cache and HBM admission (server_cache.h), host only.
// Prints "ok" and exits 0, or names the failed check and exits 1.
#include <stdio.h>
#include <vector>
#include "server_cache.h"

using helm_srv::Cache;
using helm_srv::Key;

static int failures = 0;
#define CHECK(c)                                              \
    do {                                                      \
        if (!(c)) {                                           \
            printf("FAILED line %d: %s\n", __LINE__, #c);     \
            ++failures;                                       \
        }                                                     \
    } while (0)

static void *tag(long v) { return reinterpret_cast<void *>(v); }

int main() {
    const Key A{0, 5.0, 1}, B{0, 10.0, 1}, Cc{1, 5.0, 1}, Afp64{0, 5.0, 0};
    {   // LRU order: the least recently used unpinned entry goes first
        Cache c(100);
        std::vector<void *> v;
        CHECK(c.reserve(40, &v) && v.empty());
        c.unpin(c.insert(A, 40, tag(1)));
        CHECK(c.reserve(40, &v) && v.empty());
        c.unpin(c.insert(B, 40, tag(2)));
        CHECK(c.used() == 80 && c.entries() == 2);
        helm_srv::Entry *e = c.acquire(A);   // A is now the most recent
        CHECK(e && e->payload == tag(1) && e->pins == 1);
        c.unpin(e);
        CHECK(c.reserve(40, &v));             // needs 20 more: evicts B only
        CHECK(v.size() == 1 && v[0] == tag(2));
        CHECK(c.contains(A) && !c.contains(B) && c.used() == 80 && c.evictions() == 1);
        c.release(40);
        CHECK(c.used() == 40 && c.peak() == 80);
    }
    {   // pinned entries are never evicted; an impossible reservation evicts nothing
        Cache c(100);
        std::vector<void *> v;
        c.reserve(50, &v);
        helm_srv::Entry *a = c.insert(A, 50, tag(1));   // stays pinned
        c.reserve(30, &v);
        c.unpin(c.insert(Cc, 30, tag(3)));
        CHECK(!c.can_reserve(60));
        CHECK(!c.reserve(60, &v) && v.empty() && c.contains(Cc) && c.used() == 80);
        CHECK(c.reserve(40, &v) && v.size() == 1 && v[0] == tag(3) && c.contains(A));
        CHECK(c.used() == 90);
        CHECK(!c.reserve(101, &v));   // above the budget itself
        c.unpin(a);
        CHECK(c.reserve(60, &v) && v.size() == 2 && v[1] == tag(1) && c.used() == 100);
    }
    {   // keys differ by model, frequency and precision; growth and clear
        Cache c(1000);
        std::vector<void *> v;
        c.reserve(10, &v);
        c.unpin(c.insert(A, 10, tag(1)));
        CHECK(c.acquire(Afp64) == nullptr && c.acquire(B) == nullptr && c.acquire(Cc) == nullptr);
        helm_srv::Entry *e = c.acquire(A);
        c.count(e != nullptr);
        c.count(false);
        CHECK(c.hits() == 1 && c.misses() == 1);
        c.reserve(15, &v);
        c.grow(e, 15);
        c.unpin(e);
        CHECK(e->bytes == 25 && c.resident_bytes() == 25 && c.used() == 25);
        std::vector<void *> all = c.clear();
        CHECK(all.size() == 1 && c.used() == 0 && c.entries() == 0);
    }
    if (failures) return 1;
    printf("ok\n");
    return 0;
}
