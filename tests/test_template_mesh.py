"""The shared icosphere template of the instanced forms (Sec. IV-A, second option), read from
the library on the host: a closed, outward-oriented convex mesh around the unit sphere whose
nearest face plane is at 1 + 1e-3. CPU only."""
import numpy as np
import pytest

from paper_2601_20429_gb300 import native as N


@pytest.fixture(scope="module", params=[(2, 20), (3, 80)], ids=["ico20", "ico80"])
def mesh(request):
    N.build()
    form, nf = request.param
    return N.template_mesh(form).astype(np.float64), nf


def test_closed_genus_zero_mesh(mesh):
    tri, nf = mesh
    assert tri.shape == (nf, 3, 3)
    verts, idx = np.unique(np.round(tri.reshape(-1, 3), 6), axis=0, return_inverse=True)
    faces = idx.reshape(nf, 3)
    edges = {}
    for f in faces:
        for a, b in ((f[0], f[1]), (f[1], f[2]), (f[2], f[0])):
            edges.setdefault((min(a, b), max(a, b)), []).append((a, b))
    assert all(len(v) == 2 for v in edges.values())                    # every edge in two faces
    assert all(v[0] != v[1] for v in edges.values())                   # traversed in opposite senses
    assert len(verts) - len(edges) + nf == 2                           # Euler characteristic
    r = np.linalg.norm(verts, axis=1)
    np.testing.assert_allclose(r, r[0], rtol=1e-6)                     # vertices on one sphere


def test_faces_outward_at_the_margin(mesh):
    tri, _ = mesh
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    dist = np.einsum("ij,ij->i", n, tri[:, 0])
    assert np.all(dist > 0)
    assert dist.min() == pytest.approx(1.001, abs=2e-6)


def test_every_line_through_the_unit_sphere_meets_the_mesh(mesh):
    tri, _ = mesh
    rng = np.random.default_rng(4)
    d = rng.normal(size=(3000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    # lines at distance up to 1 from the centre, starting outside the mesh
    p = rng.normal(size=(3000, 3))
    p -= np.einsum("ij,ij->i", p, d)[:, None] * d
    p *= (rng.uniform(0, 1, 3000) ** 0.5 / np.linalg.norm(p, axis=1))[:, None]
    o = p - 3.0 * d
    e1, e2 = tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]
    for oi, di in zip(o, d):
        q = np.cross(di, e2)
        det = np.einsum("ij,ij->i", e1, q)
        s = oi - tri[:, 0]
        u = np.einsum("ij,ij->i", s, q) / det
        r = np.cross(s, e1)
        v = (r @ di) / det
        ok = (u >= 0) & (v >= 0) & (u + v <= 1)
        assert ok.sum() >= 2                                           # entry and exit faces
