// Factor cache and HBM admission of the solve server (server.cu), host logic only.
//
// Every byte the server holds on the device is accounted in `used`: resident entries (an
// operator and its factor, keyed by model, frequency and precision) plus the working memory
// of the batches in flight.  reserve(b) makes room for b more bytes by evicting the least
// recently used entries that no batch is using, and refuses (evicting nothing) when even
// evicting all of them would not make room.  No CUDA here: the payload is opaque, and the
// caller frees the payloads of the evicted entries outside its lock.
#pragma once
#include <stddef.h>
#include <stdint.h>
#include <functional>
#include <unordered_map>
#include <vector>

namespace helm_srv {

struct Key {
    int32_t model;   // server model id (velocity model on its grid)
    double omega;
    int32_t prec;    // helm_prec
    bool operator==(const Key &o) const { return model == o.model && omega == o.omega && prec == o.prec; }
};

struct KeyHash {
    size_t operator()(const Key &k) const {
        const size_t h1 = std::hash<int32_t>()(k.model), h2 = std::hash<double>()(k.omega);
        const size_t h3 = std::hash<int32_t>()(k.prec);
        return h1 ^ (h2 * 0x9e3779b97f4a7c15ull) ^ (h3 << 1);
    }
};

struct Entry {
    Key key{};
    size_t bytes = 0;     // device bytes accounted to the entry
    int pins = 0;         // batches using it (never evicted while > 0)
    uint64_t last = 0;    // tick of the last use
    void *payload = nullptr;
};

class Cache {
public:
    explicit Cache(size_t budget) : budget_(budget) {}

    size_t budget() const { return budget_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t resident_bytes() const {
        size_t s = 0;
        for (const auto &kv : map_) s += kv.second.bytes;
        return s;
    }
    size_t entries() const { return map_.size(); }
    uint64_t hits() const { return hits_; }
    uint64_t misses() const { return misses_; }
    uint64_t evictions() const { return evictions_; }

    // The entry of k (touched and pinned), or nullptr.
    Entry *acquire(const Key &k) {
        auto it = map_.find(k);
        if (it == map_.end()) return nullptr;
        it->second.last = ++tick_;
        ++it->second.pins;
        return &it->second;
    }
    // Count a lookup that went ahead (acquire may be retried while waiting for room).
    void count(bool hit) { ++(hit ? hits_ : misses_); }

    // Whether b more bytes can be made to fit now (by evicting unpinned entries).
    bool can_reserve(size_t b) const {
        size_t evictable = 0;
        for (const auto &kv : map_)
            if (kv.second.pins == 0) evictable += kv.second.bytes;
        return used_ - evictable + b <= budget_ && b <= budget_;
    }

    // Make room for b more bytes and account them; the evicted entries' payloads are
    // appended to victims.  Returns false, evicting nothing, if b cannot be made to fit.
    bool reserve(size_t b, std::vector<void *> *victims) {
        if (!can_reserve(b)) return false;
        while (used_ + b > budget_) {
            auto lru = map_.end();
            for (auto it = map_.begin(); it != map_.end(); ++it)
                if (it->second.pins == 0 && (lru == map_.end() || it->second.last < lru->second.last)) lru = it;
            used_ -= lru->second.bytes;   // can_reserve guarantees an unpinned entry exists
            if (victims) victims->push_back(lru->second.payload);
            map_.erase(lru);
            ++evictions_;
        }
        used_ += b;
        if (used_ > peak_) peak_ = used_;
        return true;
    }

    // Give back b reserved bytes (working memory of a finished batch, or a failed build).
    void release(size_t b) { used_ -= b < used_ ? b : used_; }

    // New entry for k holding `bytes` that the caller has already reserved; returned pinned.
    Entry *insert(const Key &k, size_t bytes, void *payload) {
        Entry e;
        e.key = k;
        e.bytes = bytes;
        e.pins = 1;
        e.last = ++tick_;
        e.payload = payload;
        return &(map_[k] = e);
    }

    // The entry grows by extra bytes that the caller has already reserved.
    void grow(Entry *e, size_t extra) { e->bytes += extra; }

    // Whether an entry of k is resident (no touch, no pin).
    bool contains(const Key &k) const { return map_.count(k) != 0; }

    // Remove the entry of k if it is resident and unpinned; returns its payload (or nullptr).
    void *evict(const Key &k) {
        auto it = map_.find(k);
        if (it == map_.end() || it->second.pins > 0) return nullptr;
        void *p = it->second.payload;
        used_ -= it->second.bytes;
        map_.erase(it);
        ++evictions_;
        return p;
    }

    void unpin(Entry *e) {
        if (e->pins > 0) --e->pins;
    }

    // Remove every entry (all must be unpinned); returns their payloads.
    std::vector<void *> clear() {
        std::vector<void *> out;
        for (auto &kv : map_) {
            used_ -= kv.second.bytes;
            out.push_back(kv.second.payload);
        }
        map_.clear();
        return out;
    }

private:
    size_t budget_;
    size_t used_ = 0, peak_ = 0;
    uint64_t tick_ = 0, hits_ = 0, misses_ = 0, evictions_ = 0;
    std::unordered_map<Key, Entry, KeyHash> map_;
};

}  // namespace helm_srv
