// Host check of the batched launch's queue order (batch_order.hpp): every
// (transform, pass) group appears once; each pass follows its transform's
// previous pass; a later pass is separated from its predecessor by at least
// the first passes of the next block (or, in the tail, by the other
// transforms' groups of the same step); groups of one block and pass are
// contiguous.  Random batches of 1..3-pass transforms, several block sizes.
// Then the kernel's claim protocol is simulated on such orders with random
// item times and grid sizes: every run finishes.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>

#include "batch_order.hpp"

static int fails = 0;
#define CHECK(c, ...)                        \
    do {                                     \
        if (!(c)) {                          \
            if (fails < 20) {                \
                std::printf("FAIL: " __VA_ARGS__); \
                std::printf("\n");           \
            }                                \
            ++fails;                         \
        }                                    \
    } while (0)

int main() {
    std::mt19937 rng(12345);
    for (int trial = 0; trial < 400; ++trial) {
        const int count = 1 + static_cast<int>(rng() % 300);
        const size_t block = 1 + rng() % 200;
        std::vector<std::vector<size_t>> passes(count);
        for (auto& p : passes) {
            const int np = 1 + static_cast<int>(rng() % 3);
            for (int j = 0; j < np; ++j) p.push_back(1 + rng() % 64);
        }
        const auto order = qft::wavefront_order(passes, block);
        // positions (in items) of each group
        std::map<std::pair<int, int>, std::pair<size_t, size_t>> span;  // start, end
        size_t pos = 0, total = 0;
        for (const auto& tj : order) {
            CHECK(tj.first >= 0 && tj.first < count && tj.second >= 0 &&
                      tj.second < static_cast<int>(passes[tj.first].size()),
                  "trial %d: bad group (%d,%d)", trial, tj.first, tj.second);
            CHECK(!span.count(tj), "trial %d: group (%d,%d) twice", trial, tj.first, tj.second);
            const size_t n = passes[tj.first][tj.second];
            span[tj] = {pos, pos + n};
            pos += n;
        }
        for (int t = 0; t < count; ++t)
            for (size_t j = 0; j < passes[t].size(); ++j) {
                total += passes[t][j];
                CHECK(span.count({t, static_cast<int>(j)}), "trial %d: group (%d,%zu) missing", trial, t, j);
            }
        CHECK(pos == total, "trial %d: %zu items queued, %zu expected", trial, pos, total);
        // blocks as the order defines them: recompute the block of each transform
        std::vector<int> blk(count);
        {
            int b = 0;
            size_t in_block = 0;
            for (int t = 0; t < count; ++t) {
                if (in_block >= block && t > 0) {
                    ++b;
                    in_block = 0;
                }
                blk[t] = b;
                in_block += passes[t][0];
            }
        }
        const int nblocks = blk[count - 1] + 1;
        std::vector<size_t> first_items(nblocks, 0);
        for (int t = 0; t < count; ++t) first_items[blk[t]] += passes[t][0];
        for (int t = 0; t < count; ++t)
            for (size_t j = 1; j < passes[t].size(); ++j) {
                const auto prev = span[{t, static_cast<int>(j - 1)}];
                const auto cur = span[{t, static_cast<int>(j)}];
                CHECK(cur.first >= prev.second, "trial %d: pass %zu of %d before its predecessor", trial, j, t);
                if (j == 1 && blk[t] + 1 < nblocks)
                    CHECK(cur.first - prev.second >= first_items[blk[t] + 1],
                          "trial %d: pass 1 of %d only %zu items behind pass 0", trial, t, cur.first - prev.second);
            }
        // groups of one (block, pass) are contiguous in the queue
        std::map<std::pair<int, int>, std::pair<size_t, size_t>> run;  // first and last index in `order`
        for (size_t i = 0; i < order.size(); ++i) {
            const auto key = std::make_pair(blk[order[i].first], order[i].second);
            if (!run.count(key)) run[key] = {i, i};
            run[key].second = i;
        }
        for (const auto& kv : run) {
            size_t members = 0;
            for (const auto& tj : order)
                if (blk[tj.first] == kv.first.first && tj.second == kv.first.second) ++members;
            CHECK(kv.second.second - kv.second.first + 1 == members, "trial %d: block %d pass %d not contiguous",
                  trial, kv.first.first, kv.first.second);
        }
    }
    // Progress of the kernel's claim protocol on these orders: G persistent
    // CTAs claim items in queue order; while computing its current item a CTA
    // claims the next one and starts its load if the producers are done,
    // else waits for them after the current item.  Items take random times.
    // Every run must finish (the earliest unfinished item is always some
    // CTA's current item with its producers done).
    for (int trial = 0; trial < 300; ++trial) {
        const int count = 1 + static_cast<int>(rng() % 120);
        const int G = 1 + static_cast<int>(rng() % 40);
        const size_t block = 1 + rng() % (4 * static_cast<size_t>(G));
        std::vector<std::vector<size_t>> passes(count);
        for (auto& p : passes) {
            const int np = 1 + static_cast<int>(rng() % 3);
            for (int j = 0; j < np; ++j) p.push_back(1 + rng() % 16);
        }
        const auto order = qft::wavefront_order(passes, block);
        struct Item { int t, j; };
        std::vector<Item> items;
        for (const auto& tj : order)
            for (size_t k = 0; k < passes[tj.first][tj.second]; ++k) items.push_back({tj.first, tj.second});
        const int nitems = static_cast<int>(items.size());
        std::map<std::pair<int, int>, size_t> done;  // completed tiles per (transform, pass)
        auto ready = [&](int i) {
            const Item& it = items[i];
            return it.j == 0 || done[{it.t, it.j - 1}] == passes[it.t][it.j - 1];
        };
        struct Cta { int cur = -1, nx = -1, left = 0; bool waiting = false; };
        std::vector<Cta> ctas(G);
        int next = 0, finished = 0;
        for (auto& c : ctas) {  // first claims; the first load waits for its producers
            c.cur = next < nitems ? next++ : nitems;
            c.waiting = c.cur < nitems && !ready(c.cur);
        }
        long long tick = 0;
        bool stuck = false;
        while (finished < nitems) {
            bool progress = false;
            for (auto& c : ctas) {
                if (c.cur >= nitems) continue;
                if (c.waiting) {
                    if (ready(c.cur)) { c.waiting = false; progress = true; }
                    continue;
                }
                if (c.left == 0) {  // start the item: claim the next one
                    c.nx = next < nitems ? next++ : nitems;
                    c.left = 1 + static_cast<int>(rng() % 4);
                    progress = true;
                }
                if (--c.left == 0) {  // item stored: signal, move on
                    const Item& it = items[c.cur];
                    ++done[{it.t, it.j}];
                    ++finished;
                    c.cur = c.nx;
                    c.waiting = c.cur < nitems && !ready(c.cur);
                }
                progress = true;
            }
            if (!progress) { stuck = true; break; }
            if (++tick > 100000000LL) { stuck = true; break; }
        }
        CHECK(!stuck, "protocol trial %d (G=%d, %d items): no progress with %d items finished", trial, G, nitems,
              finished);
    }
    if (fails) {
        std::printf("%d failures\n", fails);
        return 1;
    }
    std::printf("ALL OK\n");
    return 0;
}
