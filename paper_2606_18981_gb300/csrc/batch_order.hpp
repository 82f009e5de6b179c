// batch_order.hpp -- queue order of a batched launch's work items (host only).
//
// A later pass's tiles wait for all tiles of the transform's previous pass;
// placed right behind them, they would be claimed while those are still being
// computed and their CTAs would idle.  So the transforms (in the given order)
// form blocks whose first passes hold at least `block_items` items, and the
// queue runs as a wavefront: step s holds pass 0 of block s, then pass 1 of
// block s - 1, pass 2 of block s - 2, ...  A later pass then follows its
// predecessor by about a block of other items (its input still in L2), and
// each CTA sees runs of items of one pass shape.  Every group follows the
// previous pass of its own transform, so every item depends only on items
// earlier in the queue, which the persistent grid's in-order claiming needs
// for progress.
#pragma once

#include <algorithm>
#include <cstddef>
#include <utility>
#include <vector>

namespace qft {

// passes[t][j] = number of tile items of pass j of transform t (every
// transform has at least one pass).  Returns the (transform, pass) groups in
// queue order; each group's items stay together.
inline std::vector<std::pair<int, int>> wavefront_order(const std::vector<std::vector<size_t>>& passes,
                                                        size_t block_items) {
    std::vector<std::vector<int>> blocks(1);
    size_t in_block = 0, max_passes = 1;
    for (int t = 0; t < static_cast<int>(passes.size()); ++t) {
        if (in_block >= block_items && !blocks.back().empty()) {
            blocks.emplace_back();
            in_block = 0;
        }
        blocks.back().push_back(t);
        in_block += passes[t][0];
        max_passes = std::max(max_passes, passes[t].size());
    }
    std::vector<std::pair<int, int>> order;
    const size_t nblocks = blocks.size();
    for (size_t step = 0; step + 1 < nblocks + max_passes; ++step)
        for (size_t j = 0; j < max_passes && j <= step; ++j) {
            if (step - j >= nblocks) continue;
            for (int t : blocks[step - j])
                if (j < passes[t].size()) order.emplace_back(t, static_cast<int>(j));
        }
    return order;
}

}  // namespace qft
