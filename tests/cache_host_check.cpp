// Host-only check of the context's cache bookkeeping (lgf_cache.h): LRU
// bounds, pinning of the running call's entries, and the rule that scratch
// growth or an eviction drops every captured graph.  Built with g++ by
// tests/test_cache_host.py; prints one line per check and exits non-zero on
// the first failure.
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <string>
#include <vector>

#include "lgf_cache.h"
#include "lgf_tune.h"

using namespace lgf;

static int g_failed = 0;
#define CHECK(cond)                                                                 \
    do {                                                                            \
        if (!(cond)) {                                                              \
            std::printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #cond);              \
            g_failed = 1;                                                           \
            return;                                                                 \
        }                                                                           \
    } while (0)

struct Item {
    int id = 0;
    uint64_t used = 0;
    static int alive;
    explicit Item(int i) : id(i) { ++alive; }
    ~Item() { --alive; }
};
int Item::alive = 0;

static Item *find_id(LruCache<Item> &c, int id, uint64_t epoch)
{
    return c.find([&](const Item &it) { return it.id == id; }, epoch);
}

static void lru_evicts_least_recent()
{
    LruCache<Item> c(3);
    uint64_t ev = 0;
    int hooks = 0;
    auto hook = [&] { ++hooks; };
    c.insert(std::make_unique<Item>(1), 1, hook, &ev);
    c.insert(std::make_unique<Item>(2), 2, hook, &ev);
    c.insert(std::make_unique<Item>(3), 3, hook, &ev);
    CHECK(c.size() == 3 && ev == 0 && hooks == 0);
    CHECK(find_id(c, 1, 4) != nullptr);               // 1 is now the most recent
    c.insert(std::make_unique<Item>(4), 5, hook, &ev);
    CHECK(c.size() == 3 && ev == 1 && hooks == 1);
    CHECK(find_id(c, 2, 6) == nullptr);               // 2 was the least recent
    CHECK(find_id(c, 1, 6) && find_id(c, 3, 6) && find_id(c, 4, 6));
    CHECK(Item::alive == 3);
    std::printf("ok lru_evicts_least_recent\n");
}

static void running_call_entries_are_pinned()
{
    LruCache<Item> c(2);
    uint64_t ev = 0;
    int hooks = 0;
    auto hook = [&] { ++hooks; };
    // one call (epoch 7) needs three plans: none may be evicted before it returns
    Item *a = c.insert(std::make_unique<Item>(1), 7, hook, &ev);
    Item *b = c.insert(std::make_unique<Item>(2), 7, hook, &ev);
    Item *d = c.insert(std::make_unique<Item>(3), 7, hook, &ev);
    CHECK(c.size() == 3 && ev == 0 && hooks == 0);
    CHECK(a->id == 1 && b->id == 2 && d->id == 3);    // pointers still valid
    // the next call inserts one more: the bound is restored
    c.insert(std::make_unique<Item>(4), 8, hook, &ev);
    CHECK(c.size() == 2 && ev == 2 && hooks == 1);
    CHECK(find_id(c, 4, 9) != nullptr);
    CHECK(Item::alive == 2);                            // evicted entries are destroyed
    std::printf("ok running_call_entries_are_pinned\n");
}

static void invalidation_drops_every_graph()
{
    GraphCache<int> g(8);
    CacheCounters cnt;
    std::vector<int> destroyed;
    auto destroy = [&](int h) { destroyed.push_back(h); };
    g.add({1, 2}, 11, 1);
    g.add({3}, 12, 2);
    CHECK(g.size() == 2 && g.find({1, 2}, 3) != nullptr && *g.find({3}, 4) == 12);
    // scratch growth: the graphs captured with the old buffers must go
    g.invalidate(destroy, &cnt);
    CHECK(g.size() == 0 && cnt.generation == 1 && cnt.graphs_dropped == 2 && destroyed.size() == 2);
    CHECK(g.find({1, 2}, 5) == nullptr);                // the batch will be captured afresh
    std::printf("ok invalidation_drops_every_graph\n");
}

static void graph_bound_evicts_least_recent()
{
    GraphCache<int> g(2);
    CacheCounters cnt;
    std::vector<int> destroyed;
    auto destroy = [&](int h) { destroyed.push_back(h); };
    g.make_room(destroy, &cnt);
    g.add({1}, 101, 1);
    g.make_room(destroy, &cnt);
    g.add({2}, 102, 2);
    CHECK(g.find({1}, 3) != nullptr);                   // {1} most recent
    g.make_room(destroy, &cnt);
    g.add({3}, 103, 4);
    CHECK(g.size() == 2 && destroyed.size() == 1 && destroyed[0] == 102 && cnt.generation == 0);
    GraphCache<int> off(0);                             // cap 0: nothing kept
    off.make_room(destroy, &cnt);
    CHECK(off.size() == 0);
    std::printf("ok graph_bound_evicts_least_recent\n");
}

static void tune_file_round_trip()
{
    const int nbs[3] = {4, 2, 4}, nbt[3] = {67, 4, 4}, off[3] = {-1, -1, 0};
    const std::string k = tune_plan_key(false, 16, nbs, nbt, off, 3);
    CHECK(k == "P f32 b16 s4,2,4 t67,4,4 o-1,-1,0 nf3");
    TuneChoiceText c;
    c.shift[0] = 1;
    c.shift[1] = 1;
    c.bump[2] = 1;
    c.zvar = 1;
    c.fuse = 1;
    const std::string v = tune_plan_value(c);
    CHECK(v == "x1 y1 bx0 by0 bz1 z1 f1");
    std::map<std::string, std::string> m;
    std::string text = "# comment\n" + tune_line(k, "x0 y0 bx0 by0 bz0 z0") + "garbage line\n" + tune_line(k, v) +
                       tune_line(tune_batch_key(true, 0x9f3aull), "nb2") + " -> lonely\n";
    CHECK(tune_parse(text, &m) == 3);
    CHECK(m.size() == 2 && m[k] == v);                      // the later line wins
    CHECK(m[tune_batch_key(true, 0x9f3aull)] == "nb2");
    TuneChoiceText r;
    CHECK(tune_parse_plan_value(m[k], &r));
    CHECK(r.shift[0] == 1 && r.shift[1] == 1 && r.bump[0] == 0 && r.bump[2] == 1 && r.zvar == 1 && r.fuse == 1);
    CHECK(tune_parse_plan_value("x0 y1 bx0 by0 bz0 z1", &r) && r.fuse == 0);   // older file: apart, the default
    CHECK(!tune_parse_plan_value("x0 y0 bx0 by0 bz0 z0 f2", &r));             // out of range
    CHECK(!tune_parse_plan_value("x2 y0 bx0 by0 bz0 z0", &r));   // out of range
    CHECK(!tune_parse_plan_value("x1 y0", &r));                  // truncated
    const unsigned char a[3] = {1, 2, 3}, b[3] = {1, 2, 4};
    CHECK(tune_hash(a, 3) != tune_hash(b, 3) && tune_hash(a, 3) == tune_hash(a, 3));
    std::printf("ok tune_file_round_trip\n");
}

int main()
{
    lru_evicts_least_recent();
    if (!g_failed) running_call_entries_are_pinned();
    if (!g_failed) invalidation_drops_every_graph();
    if (!g_failed) graph_bound_evicts_least_recent();
    if (!g_failed) tune_file_round_trip();
    return g_failed;
}
