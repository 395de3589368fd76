// Host test of the serving loop's scheduling (sx_sched.h), no GPU: the arena allocator against a
// byte-level model under random allocation and release, and the step planner's policies on
// hand-made request mixes plus invariants over random ones.  Prints "ok" and exits 0, or names
// the first failed check and exits 1.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "sx_sched.h"

using sx::sched::Arena;
using sx::sched::Want;

static int failures = 0;
#define CHECK(c)                                                         \
    do {                                                                 \
        if (!(c)) {                                                      \
            std::fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #c); \
            if (++failures > 10) std::exit(1);                           \
        }                                                                \
    } while (0)

static void arena_basics() {
    Arena a(1 << 20);
    size_t o1 = 9, o2 = 9, o3 = 9, o4 = 9;
    CHECK(a.alloc(1000, &o1) && o1 == 0);       // rounded up to 1024
    CHECK(a.alloc(1, &o2) && o2 == 1024);       // 256
    CHECK(a.alloc(0, &o3) && o3 == 1280);       // a zero-byte request still takes 256
    CHECK(a.used() == 1024 + 256 + 256);
    a.release(o2, 1);                           // a 256-byte hole at 1024
    CHECK(a.alloc(200, &o4) && o4 == 1024);     // first fit takes the hole
    a.release(o1, 1000);
    a.release(o4, 200);
    a.release(o3, 0);
    CHECK(a.used() == 0 && a.free_blocks() == 1);  // coalesced back into one block
    CHECK(a.peak() == 1024 + 256 + 256);
    size_t all = 9;
    CHECK(a.alloc(1 << 20, &all) && all == 0);
    size_t none = 9;
    CHECK(!a.alloc(1, &none));
    a.release(all, 1 << 20);
    CHECK(a.used() == 0 && a.free_blocks() == 1);
}

// Random alloc/release against a model: no two live blocks overlap, every block lies inside the
// arena and is aligned, `used` is the sum of the live rounded sizes, and once everything is
// released the free list is one block again.
static void arena_random() {
    const size_t size = 64u << 20;
    Arena a(size);
    std::mt19937_64 rng(20260603);
    struct Live { size_t off, bytes; };
    std::vector<Live> live;
    std::vector<unsigned char> owner(size / sx::sched::kAlign, 0);
    size_t used = 0;
    for (int step = 0; step < 20000; ++step) {
        if (live.empty() || rng() % 3 != 0) {
            const size_t bytes = (rng() % 4 == 0) ? rng() % (4u << 20) : rng() % 65536;
            size_t off = 0;
            if (a.alloc(bytes, &off)) {
                const size_t r = sx::sched::arena_bytes(bytes);
                CHECK(off % sx::sched::kAlign == 0 && off + r <= size);
                for (size_t u = off / sx::sched::kAlign; u < (off + r) / sx::sched::kAlign; ++u) {
                    CHECK(owner[u] == 0);
                    owner[u] = 1;
                }
                live.push_back({off, bytes});
                used += r;
            }
        } else {
            const size_t k = rng() % live.size();
            const size_t r = sx::sched::arena_bytes(live[k].bytes);
            for (size_t u = live[k].off / sx::sched::kAlign; u < (live[k].off + r) / sx::sched::kAlign; ++u) owner[u] = 0;
            a.release(live[k].off, live[k].bytes);
            used -= r;
            live[k] = live.back();
            live.pop_back();
        }
        CHECK(a.used() == used);
    }
    for (const Live &l : live) a.release(l.off, l.bytes);
    CHECK(a.used() == 0 && a.free_blocks() == 1);
}

static Want want(uint64_t key, uint64_t seq, uint64_t per, uint64_t remaining, uint64_t later) {
    return Want{key, seq, per, remaining, later};
}

static void policy_srpt() {
    // totals: key 0 = 8000*8 + 0, key 1 = 100*8 + 800 (short), key 2 = 1e6*8 (long)
    std::vector<Want> w = {want(0, 0, 8, 8000, 0), want(1, 1, 8, 100, 800), want(2, 2, 8, 1000000, 0)};
    const auto g = sx::sched::plan_step(SX_SERVE_POLICY_SRPT, 1 << 20, w);
    CHECK(w[0].key == 1 && w[1].key == 0 && w[2].key == 2);  // shortest remaining work first
    CHECK(g[0] == 100 && g[1] == 8000);                       // all of their current phase
    const uint64_t left = (1 << 20) - 100 * 8 - 8000 * 8;
    CHECK(g[2] == left / 8 / 64 * 64);                        // the rest, in whole 64-element units
    // equal totals: admission order
    std::vector<Want> t = {want(5, 9, 8, 64, 0), want(6, 3, 8, 64, 0)};
    sx::sched::plan_step(SX_SERVE_POLICY_SRPT, 4096, t);
    CHECK(t[0].key == 6);
}

static void policy_fair() {
    // budget 3 MiB over three requests: the small one gets all, the two large split the rest
    const uint64_t budget = 3u << 20;
    std::vector<Want> w = {want(0, 0, 8, 1u << 20, 0), want(1, 1, 8, 1000, 0), want(2, 2, 8, 1u << 20, 0)};
    const auto g = sx::sched::plan_step(SX_SERVE_POLICY_FAIR, budget, w);
    CHECK(w[0].key == 1 && g[0] == 1000);
    const uint64_t each = (budget - 8000) / 2 / 8 / 64 * 64;
    CHECK(g[1] == each && g[2] >= each && g[2] - each < 64 * 2);
}

static void policy_short_first() {
    const uint64_t budget = 1u << 20;  // short: total <= 256 KiB
    std::vector<Want> w = {want(0, 0, 8, 1000000, 0),         // 8 MB: long, admitted first
                           want(1, 1, 8, 20000, 0),           // 160 KB: short
                           want(2, 2, 8, 1000, 0)};           // 8 KB: short, shortest
    const auto g = sx::sched::plan_step(SX_SERVE_POLICY_SHORT_FIRST, budget, w);
    CHECK(w[0].key == 2 && w[1].key == 1 && w[2].key == 0);
    CHECK(g[0] == 1000 && g[1] == 20000);
    CHECK(g[2] == (budget - 8000 - 160000) / 8 / 64 * 64);
}

// Invariants on random mixes: a grant never exceeds what is left and is whole 64-element units
// unless it is all that is left; a step is never empty; the bytes granted exceed the budget by
// less than 64 elements' worth per request (FAIR gives every request at least 64 elements).
static void policy_random() {
    std::mt19937_64 rng(7);
    for (int trial = 0; trial < 3000; ++trial) {
        const int policy = (int)(rng() % 3);
        const uint64_t budget = (1u << 16) + rng() % (1u << 26);
        std::vector<Want> w;
        const int count = 1 + (int)(rng() % 40);
        for (int k = 0; k < count; ++k) {
            const uint64_t per = (rng() % 2 ? 8 : 4) * (1 + rng() % 3);
            const uint64_t remaining = 1 + rng() % ((rng() % 4 == 0) ? (1u << 24) : 5000);
            w.push_back(want(k, k, per, remaining, (rng() % 2) ? remaining * per : 0));
        }
        const auto g = sx::sched::plan_step(policy, budget, w);
        uint64_t bytes = 0, max_per = 0;
        bool any = false;
        for (size_t i = 0; i < w.size(); ++i) {
            CHECK(g[i] <= w[i].remaining);
            CHECK(g[i] == w[i].remaining || g[i] % 64 == 0);
            bytes += g[i] * w[i].per;
            if (g[i]) {
                any = true;
                max_per = std::max(max_per, w[i].per);
            }
        }
        CHECK(any && g[0] > 0);
        CHECK(bytes < budget + 64 * max_per * w.size());
    }
}

// Admission: arrival order; later requests pass one that does not fit until it has been passed
// kMaxBypass times, after which nothing is admitted before it; the slot limit holds; the
// look-ahead is bounded and asks for another pass when it runs out with room left.
struct FakeReq {
    int id;
    size_t bytes;
    int bypassed = 0;
};

static void admission() {
    using sx::sched::admission_pass;
    std::vector<FakeReq> reqs;
    for (int k = 0; k < 10; ++k) reqs.push_back({k, (k == 2) ? 1000u : 10u});
    std::deque<FakeReq *> waiting;
    for (auto &r : reqs) waiting.push_back(&r);
    std::vector<FakeReq *> active;
    size_t free_bytes = 100;
    auto fits = [&](FakeReq *q) {
        if (q->bytes > free_bytes) return false;
        free_bytes -= q->bytes;
        return true;
    };
    // request 2 does not fit: 0, 1 and 3..9 are admitted in order past it, and it is passed 7 times
    CHECK(!admission_pass(waiting, active, 100, fits));
    CHECK(active.size() == 9 && waiting.size() == 1 && waiting[0]->id == 2);
    CHECK(active[0]->id == 0 && active[1]->id == 1 && active[2]->id == 3);
    CHECK(reqs[2].bypassed == 7);
    // once passed kMaxBypass times, nothing gets in before it
    reqs[2].bypassed = sx::sched::kMaxBypass;
    FakeReq late{42, 1};
    waiting.push_back(&late);
    CHECK(!admission_pass(waiting, active, 100, fits));
    CHECK(waiting.size() == 2 && waiting[1]->id == 42);
    free_bytes = 2000;  // now it fits, and the late one follows in order
    CHECK(!admission_pass(waiting, active, 100, fits));
    CHECK(waiting.empty() && active[active.size() - 2]->id == 2 && active.back()->id == 42);
    // slot limit
    std::vector<FakeReq> many(10, FakeReq{0, 1});
    std::deque<FakeReq *> w2;
    for (auto &r : many) w2.push_back(&r);
    std::vector<FakeReq *> a2;
    free_bytes = 1000;
    CHECK(!admission_pass(w2, a2, 4, fits));
    CHECK(a2.size() == 4 && w2.size() == 6);
    // bounded look-ahead: 200 requests that do not fit ahead of one that does
    std::vector<FakeReq> big(200, FakeReq{1, 1u << 30});
    FakeReq small{2, 1};
    std::deque<FakeReq *> w3;
    for (auto &r : big) w3.push_back(&r);
    w3.push_back(&small);
    std::vector<FakeReq *> a3;
    CHECK(admission_pass(w3, a3, 100, fits));  // ran out of look-ahead: try again
    CHECK(a3.empty() && w3.size() == 201);
}

int main() {
    admission();
    arena_basics();
    arena_random();
    policy_srpt();
    policy_fair();
    policy_short_first();
    policy_random();
    if (failures) return 1;
    std::printf("ok\n");
    return 0;
}
