// Host-side cache bookkeeping of a context: plan caches with a bounded,
// least-recently-used size, and the rule that ties captured CUDA graphs to the
// buffers they were captured with.  Plain C++ (no CUDA): the library uses it,
// and the host tests compile it alone.
//
// Two hazards it removes:
//   - A captured graph bakes in the device pointers of the scratch buffers,
//     plans and spectra that were current at capture.  Whenever any of them is
//     freed or reallocated (scratch growth, plan or spectrum eviction, table
//     rebuild) every cached graph is dropped, so no replay can touch freed
//     memory.  `generation` counts these events.
//   - An adaptive active set changes from step to step, so plans keyed by
//     block lists would accumulate without bound.  Each cache keeps at most
//     `cap` entries; the entries used by the current public call (stamp equal
//     to the call's epoch) are never evicted, so a batch with more distinct
//     plans than `cap` still finds all of its plans alive until it returns.
#pragma once
#include <cstddef>
#include <cstdint>
#include <memory>
#include <vector>

namespace lgf {

// Counters reported through lgf_ctx_stats.
struct CacheCounters {
    uint64_t epoch = 1;              // public calls entered
    uint64_t generation = 0;         // invalidations of the captured graphs
    uint64_t graphs_dropped = 0;     // graphs destroyed by invalidation or LRU
    uint64_t plans_evicted = 0;      // plans and spectra released by the LRU bound
    uint64_t scratch_reallocs = 0;   // scratch buffers (re)allocated
};

// A vector of owned entries, each with a `used` stamp.  T must have a public
// member `uint64_t used`.
template <class T>
class LruCache {
public:
    explicit LruCache(size_t cap = 256) : cap_(cap) {}

    size_t size() const { return items_.size(); }
    size_t cap() const { return cap_; }
    void set_cap(size_t cap) { cap_ = cap < 1 ? 1 : cap; }
    void clear() { items_.clear(); }

    // First entry matching `pred`, stamped with `epoch`; nullptr if none.
    template <class Pred>
    T *find(Pred pred, uint64_t epoch)
    {
        for (auto &p : items_)
            if (pred(*p)) {
                p->used = epoch;
                return p.get();
            }
        return nullptr;
    }

    // Number of entries that insert() would evict to stay within the bound
    // (entries stamped with `epoch` are pinned).
    size_t would_evict(uint64_t epoch) const
    {
        size_t unpinned = 0;
        for (auto &p : items_) unpinned += p->used != epoch;
        const size_t over = items_.size() + 1 > cap_ ? items_.size() + 1 - cap_ : 0;
        return over < unpinned ? over : unpinned;
    }

    // Insert `item` stamped with `epoch` after evicting the least recently
    // used unpinned entries beyond the bound.  `before_evict()` runs once,
    // before the first eviction (the caller drops graphs and synchronises
    // there); evicted entries are destroyed after it.  Returns the inserted
    // entry and adds the number evicted to *evicted.
    template <class BeforeEvict>
    T *insert(std::unique_ptr<T> item, uint64_t epoch, BeforeEvict before_evict, uint64_t *evicted)
    {
        size_t n = would_evict(epoch);
        if (n > 0) {
            before_evict();
            while (n-- > 0) {
                size_t lru = items_.size();
                for (size_t i = 0; i < items_.size(); ++i)
                    if (items_[i]->used != epoch && (lru == items_.size() || items_[i]->used < items_[lru]->used))
                        lru = i;
                if (lru == items_.size()) break;
                items_.erase(items_.begin() + (std::ptrdiff_t)lru);
                if (evicted) ++*evicted;
            }
        }
        item->used = epoch;
        items_.push_back(std::move(item));
        return items_.back().get();
    }

    // Destroy every entry matching `pred` (the caller has made sure nothing
    // in flight or captured still uses them).
    template <class Pred>
    size_t erase_if(Pred pred)
    {
        size_t n = 0;
        for (size_t i = items_.size(); i-- > 0;)
            if (pred(*items_[i])) {
                items_.erase(items_.begin() + (std::ptrdiff_t)i);
                ++n;
            }
        return n;
    }

    std::vector<std::unique_ptr<T>> &items() { return items_; }

private:
    size_t cap_;
    std::vector<std::unique_ptr<T>> items_;
};

// Graph cache entry: byte key plus an opaque executable handle.
template <class Exec>
struct GraphSlot {
    std::vector<unsigned char> key;
    Exec exec{};
    uint64_t used = 0;
};

// Keyed graph cache with an LRU bound; `destroy(exec)` releases a handle.
template <class Exec>
class GraphCache {
public:
    explicit GraphCache(size_t cap = 8) : cap_(cap) {}
    size_t size() const { return slots_.size(); }
    size_t cap() const { return cap_; }
    void set_cap(size_t cap) { cap_ = cap; }

    Exec *find(const std::vector<unsigned char> &key, uint64_t stamp)
    {
        for (auto &g : slots_)
            if (g.key == key) {
                g.used = stamp;
                return &g.exec;
            }
        return nullptr;
    }

    // Make room for one more graph (cap 0: nothing is cached).
    template <class Destroy>
    void make_room(Destroy destroy, CacheCounters *c)
    {
        while (!slots_.empty() && slots_.size() + 1 > cap_) {
            size_t lru = 0;
            for (size_t i = 1; i < slots_.size(); ++i)
                if (slots_[i].used < slots_[lru].used) lru = i;
            destroy(slots_[lru].exec);
            slots_.erase(slots_.begin() + (std::ptrdiff_t)lru);
            if (c) ++c->graphs_dropped;
        }
    }

    void add(std::vector<unsigned char> key, Exec exec, uint64_t stamp)
    {
        GraphSlot<Exec> s;
        s.key = std::move(key);
        s.exec = exec;
        s.used = stamp;
        slots_.push_back(std::move(s));
    }

    // Drop every graph: the buffers they were captured with are about to be
    // freed or replaced.
    template <class Destroy>
    void invalidate(Destroy destroy, CacheCounters *c)
    {
        for (auto &g : slots_) destroy(g.exec);
        if (c) {
            c->graphs_dropped += slots_.size();
            ++c->generation;
        }
        slots_.clear();
    }

private:
    size_t cap_;
    std::vector<GraphSlot<Exec>> slots_;
};

}  // namespace lgf
