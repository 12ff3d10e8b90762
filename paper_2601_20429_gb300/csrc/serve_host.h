// Host-only scheduling logic of the request server (no CUDA types, so that it is also built and
// tested on its own): the first-fit output arena, the choice of the work published next, the
// regrouping of untraced tiles into ranges, and the division of a memory budget.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <algorithm>
#include <deque>
#include <iterator>
#include <map>
#include <utility>
#include <vector>

namespace grtx_serve {

// First-fit allocator over the output arena (offsets on the host, 256-byte granules).
struct Arena {
    char *base = nullptr;
    size_t bytes = 0, used = 0;
    std::map<size_t, size_t> free_;     // offset -> size, coalesced
    std::map<size_t, size_t> live;      // offset -> size of outputs handed out
    void reset(char *b, size_t n)
    {
        base = b;
        bytes = n;
        used = 0;
        free_.clear();
        live.clear();
        if (n) free_[0] = n;
    }
    static size_t round(size_t n) { return (n + 255) / 256 * 256; }
    char *alloc(size_t n)
    {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            size_t off = it->first, sz = it->second;
            free_.erase(it);
            if (sz > n) free_[off + n] = sz - n;
            live[off] = n;
            used += n;
            return base + off;
        }
        return nullptr;
    }
    bool release(char *p)
    {
        if (!base || p < base || p >= base + bytes) return false;
        auto it = live.find((size_t)(p - base));
        if (it == live.end()) return false;
        size_t off = it->first, n = it->second;
        live.erase(it);
        used -= n;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + n == nx->first) {      // merge with the next free block
            n += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {                              // and with the previous one
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += n;
                return true;
            }
        }
        free_[off] = n;
        return true;
    }
};

// A piece of a request published to a launch: items [begin, begin + count) of request r.
template <class Req>
struct Piece {
    Req *r;
    unsigned begin, count;
};

// Unscheduled work, up to `budget` items (a multiple of 32) and `max_pieces` pieces, request by
// request in order of deadline: admission time plus size_ns per ray of the whole request (0:
// admission order; large: smallest request first; admission order among equal deadlines). A
// request's ranges that a launch did not trace come first, then its next items. Req has
// n_items, next (first item not yet published), retry (a vector of {first item, count}) and
// t_admit; next and retry are advanced past what is taken.
template <class Req, class Active>
std::vector<Piece<Req>> take_pieces(const Active &active, double size_ns, int64_t budget, int max_pieces)
{
    std::vector<std::pair<double, Req *>> order;
    for (Req *r : active) {
        if (r->next >= r->n_items && r->retry.empty()) continue;
        order.push_back({r->t_admit + 1e-9 * size_ns * (double)r->n_items, r});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<double, Req *> &x, const std::pair<double, Req *> &y) {
                         return x.first < y.first;
                     });
    std::vector<Piece<Req>> pieces;
    for (const auto &o : order) {
        Req *r = o.second;
        while (!r->retry.empty() && budget > 0 && (int)pieces.size() < max_pieces) {
            auto &rg = r->retry.back();
            const unsigned take = (unsigned)std::min<int64_t>(rg.second, budget);
            pieces.push_back({r, rg.first, take});
            rg.first += take;
            rg.second -= take;
            if (rg.second == 0) r->retry.pop_back();
            budget -= take;
        }
        if (r->next >= r->n_items || budget <= 0 || (int)pieces.size() >= max_pieces) continue;
        unsigned take = (unsigned)std::min<int64_t>((int64_t)(r->n_items - r->next), budget);
        pieces.push_back({r, r->next, take});
        r->next += take;
        budget -= take;
    }
    return pieces;
}

// Untraced 32-item tiles {request, first item} of an ended launch, given back to their
// requests' retry lists as ranges of consecutive items (one range per run of adjacent tiles of
// a request). Returns the number of tiles.
template <class Req>
size_t give_back_tiles(std::vector<std::pair<Req *, unsigned>> &tiles)
{
    std::sort(tiles.begin(), tiles.end());
    for (size_t i = 0; i < tiles.size();) {
        size_t e = i + 1;
        while (e < tiles.size() && tiles[e].first == tiles[i].first && tiles[e].second == tiles[e - 1].second + 32) ++e;
        tiles[i].first->retry.push_back({tiles[i].second, (unsigned)(32 * (e - i))});
        i = e;
    }
    return tiles.size();
}

// Device memory of a server under a budget (0: none). The step slots' lists take at most half
// of the budget: as many full-residency slots as fit (1 to max_steps), else one slot of as
// many 128-ray blocks as fit; the small tables (table_fixed + per slot table_per_step +
// table_per_block per block) come next, and the rest, in 256-byte granules, is the output
// arena. fits is false when not even one block of lists fits in half the budget
// (below_one_block) or the lists and tables exceed it.
struct BudgetPlan {
    int n_steps = 0, blocks = 0;
    size_t lists = 0, tables = 0, arena = 0;
    bool fits = false, below_one_block = false;
};

inline BudgetPlan plan_budget(size_t budget, int max_steps, int blocks_full, size_t per_block, size_t table_fixed,
                              size_t table_per_step, size_t table_per_block)
{
    BudgetPlan pl;
    auto tables = [&](int steps, int blocks) {
        return table_fixed + (size_t)steps * (table_per_step + table_per_block * (size_t)blocks);
    };
    if (budget == 0) {
        pl.n_steps = max_steps;
        pl.blocks = blocks_full;
        pl.lists = (size_t)max_steps * blocks_full * per_block;
        pl.tables = tables(max_steps, blocks_full);
        pl.fits = true;
        return pl;
    }
    const size_t list_cap = budget / 2;
    const size_t full_step = (size_t)blocks_full * per_block;
    pl.n_steps = (int)std::min<size_t>((size_t)max_steps, std::max<size_t>(1, list_cap / full_step));
    pl.blocks = (int)std::min<size_t>((size_t)blocks_full, list_cap / ((size_t)pl.n_steps * per_block));
    if (pl.blocks < 1) {
        pl.below_one_block = true;
        return pl;
    }
    pl.lists = (size_t)pl.n_steps * pl.blocks * per_block;
    pl.tables = tables(pl.n_steps, pl.blocks);
    if (pl.lists + pl.tables > budget) return pl;
    pl.arena = (budget - pl.lists - pl.tables) / 256 * 256;
    pl.fits = true;
    return pl;
}

}  // namespace grtx_serve
