"""The request server's host-only scheduling logic (csrc/serve_host.h), built with the host C++
compiler and run on the CPU: the deadline order of the work published next, budgets and
piece counts, ranges a launch did not trace going first, the regrouping of untraced tiles into
ranges, the first-fit output arena with coalescing, and the division of a memory budget into
step slots, tables and the arena."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_20429_gb300", "csrc")

DRIVER = r'''
#include "serve_host.h"
#include <cstdio>
#include <deque>
#include <string>
#include <vector>

using namespace grtx_serve;

struct Req {
    unsigned n_items = 0, next = 0;
    double t_admit = 0;
    std::vector<std::pair<unsigned, unsigned>> retry;
};

static int failures = 0;
#define CHECK(c) do { if (!(c)) { std::printf("FAIL line %d: %s\n", __LINE__, #c); ++failures; } } while (0)

int main()
{
    // deadline order: admission time + size_ns per ray of the whole request
    {
        Req big{100000, 0, 0.000}, small{4096, 0, 0.001};
        std::deque<Req *> active{&big, &small};
        auto p = take_pieces<Req>(active, 0.0, 1 << 20, 16);            // admission order
        CHECK(p.size() == 2 && p[0].r == &big && p[1].r == &small);
        big.next = small.next = 0;
        p = take_pieces<Req>(active, 10.0, 1 << 20, 16);                // deadlines 1.0 ms vs 1.04 ms
        CHECK(p.size() == 2 && p[0].r == &big && p[1].r == &small);
        big.next = small.next = 0;
        p = take_pieces<Req>(active, 100.0, 1 << 20, 16);               // 10 ms vs 1.41 ms: small first
        CHECK(p.size() == 2 && p[0].r == &small && p[1].r == &big);
        CHECK(p[0].begin == 0 && p[0].count == 4096 && p[1].count == 100000);
        CHECK(big.next == 100000 && small.next == 4096);
        // nothing left: no pieces
        CHECK(take_pieces<Req>(active, 100.0, 1 << 20, 16).empty());
    }
    // the budget splits a request; the rest comes in the next call, where it left off
    {
        Req r{1000 * 32, 0, 0.0};
        std::deque<Req *> active{&r};
        auto p = take_pieces<Req>(active, 5.0, 320, 16);
        CHECK(p.size() == 1 && p[0].begin == 0 && p[0].count == 320 && r.next == 320);
        p = take_pieces<Req>(active, 5.0, 1 << 20, 16);
        CHECK(p.size() == 1 && p[0].begin == 320 && p[0].count == 32000 - 320 && r.next == 32000);
    }
    // piece count limit: requests past it wait
    {
        Req a{64, 0, 0.0}, b{64, 0, 0.1}, c{64, 0, 0.2};
        std::deque<Req *> active{&a, &b, &c};
        auto p = take_pieces<Req>(active, 0.0, 1 << 20, 2);
        CHECK(p.size() == 2 && p[0].r == &a && p[1].r == &b && c.next == 0);
    }
    // untraced ranges of a request go before its next items, and are split by the budget
    {
        Req r{3200, 1600, 0.0};
        r.retry.push_back({64, 96});
        std::deque<Req *> active{&r};
        auto p = take_pieces<Req>(active, 5.0, 64, 16);
        CHECK(p.size() == 1 && p[0].begin == 64 && p[0].count == 64);
        CHECK(r.retry.size() == 1 && r.retry[0].first == 128 && r.retry[0].second == 32 && r.next == 1600);
        p = take_pieces<Req>(active, 5.0, 1 << 20, 16);
        CHECK(p.size() == 2 && p[0].begin == 128 && p[0].count == 32 && p[1].begin == 1600 && p[1].count == 1600);
        CHECK(r.retry.empty() && r.next == 3200);
    }
    // a request with only untraced ranges left is still chosen
    {
        Req r{64, 64, 0.0};
        r.retry.push_back({0, 32});
        std::deque<Req *> active{&r};
        auto p = take_pieces<Req>(active, 5.0, 1 << 20, 16);
        CHECK(p.size() == 1 && p[0].begin == 0 && p[0].count == 32 && r.retry.empty());
    }
    // untraced tiles regroup into ranges of adjacent tiles, per request, in any input order
    {
        Req r1{4096, 4096, 0.0}, r2{4096, 4096, 0.0};
        std::vector<std::pair<Req *, unsigned>> tiles{{&r1, 96}, {&r2, 0}, {&r1, 0}, {&r1, 32}, {&r1, 160}, {&r1, 128}};
        CHECK(give_back_tiles(tiles) == 6);
        // r1: 0, 32 | 96, 128, 160 ; r2: 0
        CHECK(r1.retry.size() == 2 && r2.retry.size() == 1);
        bool a = false, b = false;
        for (auto &g : r1.retry) {
            a = a || (g.first == 0 && g.second == 64);
            b = b || (g.first == 96 && g.second == 96);
        }
        CHECK(a && b);
        CHECK(r2.retry[0].first == 0 && r2.retry[0].second == 32);
    }
    // arena: 256-byte granules, first fit, coalescing in both directions, bad releases refused
    {
        static char mem[4096];
        Arena ar;
        ar.reset(mem, 4096);
        char *x = ar.alloc(100), *y = ar.alloc(300), *z = ar.alloc(256);
        CHECK(x == mem && y == mem + 256 && z == mem + 768 && ar.used == 1024);
        CHECK(!ar.release(mem + 10) && !ar.release(mem + 8192) && !ar.release(nullptr));
        CHECK(ar.release(y) && ar.used == 512);
        CHECK(!ar.release(y));                                           // twice
        char *w = ar.alloc(512);                                          // fits y's hole exactly
        CHECK(w == mem + 256);
        CHECK(ar.release(w) && ar.release(x) && ar.release(z) && ar.used == 0);
        CHECK(ar.free_.size() == 1 && ar.free_.begin()->first == 0 && ar.free_.begin()->second == 4096);
        CHECK(ar.alloc(4096) == mem && ar.alloc(1) == nullptr);
    }
    // budget plans: 64 KiB blocks of lists, 1216 blocks a full slot, up to 2 slots
    {
        const size_t blk = 65536, fixed = 256, per_step = 264 * 32 + 16, per_blk = 16;
        BudgetPlan none = plan_budget(0, 2, 1216, blk, fixed, per_step, per_blk);
        CHECK(none.fits && none.n_steps == 2 && none.blocks == 1216 && none.arena == 0);
        CHECK(none.lists == 2 * 1216 * blk);
        // one block of lists (its half holds one block, not two) and one 64 KiB output
        const size_t b1 = blk + 65536 + 16384;
        BudgetPlan p1 = plan_budget(b1, 2, 1216, blk, fixed, per_step, per_blk);
        CHECK(p1.fits && p1.n_steps == 1 && p1.blocks == 1 && p1.lists == blk);
        CHECK(p1.tables == fixed + per_step + per_blk && p1.arena % 256 == 0);
        CHECK(p1.arena >= 65536 && p1.arena < 2 * 65536 && p1.lists + p1.tables + p1.arena <= b1);
        // half the budget holds one full slot but not two: one full slot
        BudgetPlan pf = plan_budget(3 * 1216 * blk, 2, 1216, blk, fixed, per_step, per_blk);
        CHECK(pf.fits && pf.n_steps == 1 && pf.blocks == 1216);
        // room for two full slots
        BudgetPlan p2 = plan_budget(5 * 1216 * blk, 2, 1216, blk, fixed, per_step, per_blk);
        CHECK(p2.fits && p2.n_steps == 2 && p2.blocks == 1216 && p2.lists + p2.tables + p2.arena <= 5 * 1216 * blk);
        // below one block in half the budget
        BudgetPlan pb = plan_budget(blk, 2, 1216, blk, fixed, per_step, per_blk);
        CHECK(!pb.fits && pb.below_one_block);
        // lists fit in half but the tables do not fit beside them
        BudgetPlan pt = plan_budget(2 * blk, 2, 1216, blk, fixed, 2 * blk, per_blk);
        CHECK(!pt.fits && !pt.below_one_block);
    }
    if (failures) return 1;
    std::printf("ok\n");
    return 0;
}
'''


def test_serve_host_logic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "serve_host_test.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "serve_host_test"
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout + res.stderr
    assert res.stdout.strip() == "ok"
