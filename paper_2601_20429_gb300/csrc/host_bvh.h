// A BVH2 built on the host over a few boxes (the icosphere template's triangles, the
// instances of a world), in the node format of the device BVH: per node 16 floats = child 0
// box (lo xyz, hi xyz), child 1 box, the two child references as uint32 bits (bit 31: leaf,
// low bits: the box's index), and two zero floats. Node 0 is the root. Median split of the
// box centres along the widest axis; with a single box the root has one child and the
// other reference is 0xFFFFFFFF.
#pragma once

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace host_bvh {

using Box = std::array<float, 6>;
using Node = std::array<float, 16>;

inline Box empty_box() { return {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY}; }

inline void grow(Box &a, const Box &b)
{
    for (int k = 0; k < 3; ++k) {
        a[k] = std::min(a[k], b[k]);
        a[3 + k] = std::max(a[3 + k], b[3 + k]);
    }
}

struct Builder {
    const std::vector<Box> &boxes;
    std::vector<Node> nodes;
    int depth = 0;

    static void put_ref(Node &nd, int slot, uint32_t ref) { std::memcpy(&nd[12 + slot], &ref, 4); }

    // Subtree over ids[b, e): returns its reference and box.
    uint32_t build(std::vector<int> &ids, int b, int e, Box &box, int level)
    {
        depth = std::max(depth, level);
        if (e - b == 1) {
            box = boxes[ids[b]];
            return 0x80000000u | (uint32_t)ids[b];
        }
        Box cb = empty_box();
        for (int i = b; i < e; ++i) {
            const Box &x = boxes[ids[i]];
            Box c = {0.5f * (x[0] + x[3]), 0.5f * (x[1] + x[4]), 0.5f * (x[2] + x[5]),
                     0.5f * (x[0] + x[3]), 0.5f * (x[1] + x[4]), 0.5f * (x[2] + x[5])};
            grow(cb, c);
        }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (cb[3 + a] - cb[a] > cb[3 + axis] - cb[axis]) axis = a;
        int m = (b + e) / 2;
        std::nth_element(ids.begin() + b, ids.begin() + m, ids.begin() + e, [&](int x, int y) {
            return boxes[x][axis] + boxes[x][3 + axis] < boxes[y][axis] + boxes[y][3 + axis];
        });
        uint32_t me = (uint32_t)nodes.size();
        nodes.push_back({});
        Box b0 = empty_box(), b1 = empty_box();
        uint32_t r0 = build(ids, b, m, b0, level + 1);
        uint32_t r1 = build(ids, m, e, b1, level + 1);
        Node &nd = nodes[me];
        for (int k = 0; k < 6; ++k) {
            nd[k] = b0[k];
            nd[6 + k] = b1[k];
        }
        put_ref(nd, 0, r0);
        put_ref(nd, 1, r1);
        nd[14] = nd[15] = 0.f;
        box = b0;
        grow(box, b1);
        return me;
    }
};

// Nodes over boxes (n >= 1); *depth receives the tree depth in nodes on the longest path.
inline std::vector<Node> build(const std::vector<Box> &boxes, int *depth)
{
    Builder b{boxes, {}, 0};
    if (boxes.size() == 1) {
        Node nd{};
        for (int k = 0; k < 6; ++k) {
            nd[k] = boxes[0][k];
            nd[6 + k] = boxes[0][k];
        }
        Builder::put_ref(nd, 0, 0x80000000u);
        Builder::put_ref(nd, 1, 0xFFFFFFFFu);
        if (depth) *depth = 1;
        return {nd};
    }
    std::vector<int> ids(boxes.size());
    for (size_t i = 0; i < ids.size(); ++i) ids[i] = (int)i;
    Box root = empty_box();
    b.build(ids, 0, (int)ids.size(), root, 1);
    if (depth) *depth = b.depth;
    return b.nodes;
}

}  // namespace host_bvh
