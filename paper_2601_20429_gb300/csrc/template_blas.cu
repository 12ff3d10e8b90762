// The shared bottom-level structure of the instanced-icosphere forms (Sec. IV-A "Bounding
// Primitives for Gaussians", second option): one template mesh around the unit sphere -- a
// regular icosahedron (20 triangles) or its once-subdivided icosphere (80 triangles) -- with a
// small BVH over its triangles, built on the host once and kept on every device that uses
// it. Every Gaussian instance of a scene refers to the same template; at a top-level leaf the
// ray is taken into the Gaussian's unit-sphere space and traverses this BVH.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "grtx_internal.cuh"
#include "host_bvh.h"

namespace {

using V3 = std::array<double, 3>;
using F3 = std::array<int, 3>;

V3 sub(const V3 &a, const V3 &b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
V3 cross(const V3 &a, const V3 &b)
{
    return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
double dot(const V3 &a, const V3 &b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
V3 unit(const V3 &a)
{
    double l = std::sqrt(dot(a, a));
    return {a[0] / l, a[1] / l, a[2] / l};
}

struct Mesh {
    std::vector<V3> v;
    std::vector<F3> f;
};

// Regular icosahedron on the unit sphere: the 12 cyclic permutations of (0, +-1, +-phi); the
// faces are the vertex triples at pairwise edge length, oriented outwards.
Mesh icosahedron()
{
    const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
    Mesh m;
    for (int s1 = -1; s1 <= 1; s1 += 2)
        for (int s2 = -1; s2 <= 1; s2 += 2) {
            m.v.push_back({0.0, (double)s1, s2 * phi});
            m.v.push_back({(double)s1, s2 * phi, 0.0});
            m.v.push_back({s2 * phi, 0.0, (double)s1});
        }
    auto d2 = [&](int a, int b) { V3 e = sub(m.v[a], m.v[b]); return dot(e, e); };
    for (int a = 0; a < 12; ++a)
        for (int b = a + 1; b < 12; ++b)
            for (int c = b + 1; c < 12; ++c)
                if (std::fabs(d2(a, b) - 4) < 1e-9 && std::fabs(d2(b, c) - 4) < 1e-9 && std::fabs(d2(a, c) - 4) < 1e-9)
                    m.f.push_back({a, b, c});
    for (auto &x : m.v) x = unit(x);
    return m;
}

// Split every triangle into four at its edge midpoints, pushed out to the unit sphere.
Mesh subdivide(const Mesh &in)
{
    Mesh m;
    m.v = in.v;
    std::map<std::pair<int, int>, int> mid;
    auto midpoint = [&](int a, int b) {
        auto key = std::make_pair(std::min(a, b), std::max(a, b));
        auto it = mid.find(key);
        if (it != mid.end()) return it->second;
        const V3 &p = m.v[a], &q = m.v[b];
        m.v.push_back(unit({p[0] + q[0], p[1] + q[1], p[2] + q[2]}));
        int id = (int)m.v.size() - 1;
        mid[key] = id;
        return id;
    };
    for (const F3 &t : in.f) {
        int ab = midpoint(t[0], t[1]), bc = midpoint(t[1], t[2]), ca = midpoint(t[2], t[0]);
        m.f.push_back({t[0], ab, ca});
        m.f.push_back({t[1], bc, ab});
        m.f.push_back({t[2], ca, bc});
        m.f.push_back({ab, bc, ca});
    }
    return m;
}

// Orient every face outwards and scale the mesh so that its nearest face plane is at
// 1 + 1e-3 from the centre: it encloses the unit sphere with a margin.
void finish(Mesh &m)
{
    double dmin = 1e300;
    for (F3 &t : m.f) {
        V3 n = cross(sub(m.v[t[1]], m.v[t[0]]), sub(m.v[t[2]], m.v[t[0]]));
        if (dot(n, m.v[t[0]]) < 0) std::swap(t[1], t[2]);
        n = unit(cross(sub(m.v[t[1]], m.v[t[0]]), sub(m.v[t[2]], m.v[t[0]])));
        dmin = std::min(dmin, dot(n, m.v[t[0]]));
    }
    double s = (1.0 + 1e-3) / dmin;
    for (V3 &x : m.v) x = {x[0] * s, x[1] * s, x[2] * s};
}

Mesh template_mesh(int form)
{
    Mesh m = icosahedron();
    if (form == GRTX_FORM_ICO80) m = subdivide(m);
    finish(m);
    return m;
}

struct DeviceTemplate {
    float4 *nodes = nullptr, *tris = nullptr;
    int n_nodes = 0, n_tris = 0;
};

constexpr int kMaxDevices = 64;
DeviceTemplate g_tpl[kMaxDevices][2];
std::mutex g_tpl_mutex;

std::vector<std::array<float, 9>> template_triangles(int form)
{
    Mesh m = template_mesh(form);
    std::vector<std::array<float, 9>> tri(m.f.size());
    for (size_t i = 0; i < m.f.size(); ++i)
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) tri[i][3 * k + a] = (float)m.v[m.f[i][k]][a];
    return tri;
}

}  // namespace

// Device copy of the template BVH and triangles of an instanced-icosphere form on the current
// device, built on first use and kept until the process exits.
int grtx_template_blas(int form, const float4 **nodes, const float4 **tris)
{
    if (form != GRTX_FORM_ICO20 && form != GRTX_FORM_ICO80) return grtx_fail(GRTX_ERR_INVALID_ARG, "not an icosphere form");
    int dev = 0;
    GRTX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return grtx_fail(GRTX_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_tpl_mutex);
    DeviceTemplate &t = g_tpl[dev][form == GRTX_FORM_ICO80];
    if (!t.nodes) {
        std::vector<std::array<float, 9>> tri = template_triangles(form);
        std::vector<host_bvh::Box> boxes(tri.size(), host_bvh::empty_box());
        for (size_t i = 0; i < tri.size(); ++i)
            for (int k = 0; k < 3; ++k)
                host_bvh::grow(boxes[i], {tri[i][3 * k], tri[i][3 * k + 1], tri[i][3 * k + 2], tri[i][3 * k],
                                          tri[i][3 * k + 1], tri[i][3 * k + 2]});
        std::vector<host_bvh::Node> nodes = host_bvh::build(boxes, nullptr);
        std::vector<float4> hn(nodes.size() * 4), ht(tri.size() * 3);
        std::memcpy(hn.data(), nodes.data(), hn.size() * sizeof(float4));
        for (size_t i = 0; i < tri.size(); ++i)
            for (int k = 0; k < 3; ++k) ht[3 * i + k] = make_float4(tri[i][3 * k], tri[i][3 * k + 1], tri[i][3 * k + 2], 0.f);
        float4 *dn = nullptr, *dt = nullptr;
        GRTX_CUDA(cudaMalloc(&dn, hn.size() * sizeof(float4)));
        cudaError_t e = cudaMalloc(&dt, ht.size() * sizeof(float4));
        if (e != cudaSuccess) {
            cudaFree(dn);
            return grtx_cuda_fail(e, "cudaMalloc(template triangles)");
        }
        GRTX_CUDA(cudaMemcpy(dn, hn.data(), hn.size() * sizeof(float4), cudaMemcpyHostToDevice));
        GRTX_CUDA(cudaMemcpy(dt, ht.data(), ht.size() * sizeof(float4), cudaMemcpyHostToDevice));
        t.nodes = dn;
        t.tris = dt;
        t.n_nodes = (int)nodes.size();
        t.n_tris = (int)tri.size();
    }
    *nodes = t.nodes;
    *tris = t.tris;
    return GRTX_OK;
}

extern "C" GRTX_API int grtx_template_mesh(int form, float *h_tris, int *n_tris)
{
    if (!n_tris) return grtx_fail(GRTX_ERR_INVALID_ARG, "n_tris is NULL");
    if (form != GRTX_FORM_ICO20 && form != GRTX_FORM_ICO80) return grtx_fail(GRTX_ERR_INVALID_ARG, "not an icosphere form");
    std::vector<std::array<float, 9>> tri = template_triangles(form);
    *n_tris = (int)tri.size();
    if (h_tris)
        for (size_t i = 0; i < tri.size(); ++i)
            for (int k = 0; k < 9; ++k) h_tris[9 * i + k] = tri[i][k];
    return GRTX_OK;
}
