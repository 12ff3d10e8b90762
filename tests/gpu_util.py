"""Helpers shared by the GPU parity tests: comparison of GPU outputs with the FP64 oracle."""
import math

import numpy as np

ALPHA_MIN = 0.01
T_MIN = 1e-3
RGB_TOL = 2e-4          # max abs per RGB channel (and on T)
# Per-element gradient tolerance, in units of the oracle's term scale of the element (the
# summed magnitudes of its terms): about 840 FP32 unit roundoffs (2^-24). The kernel forms
# each term from FP32 values that carry a few roundoffs each, except the opacity derivative's
# colour behind a hit, a difference of two FP32 composites of up to ~100 terms, and the
# backward sums the terms with FP32 atomics.
GRAD_TERM_TOL = 5e-5


def oracle_rays_subset(rays, idx):
    return tuple(np.ascontiguousarray(a[idx]) for a in rays)


def excused_mismatch(S, ro, rd, gpu, ora, alpha_min=ALPHA_MIN, T_min=T_MIN):
    """True if two blend lists of one ray differ only where FP32 vs FP64 may legitimately
    decide differently: a hit whose alpha is within 1e-5 of alpha_min, a tail cut where the
    transmittance is within 1e-3 relative of T_min, or an order swap of near-equal depths."""
    sg, so = set(gpu), set(ora)
    for g in sg ^ so:
        t, d2, al = S.response(int(g), ro, rd)
        if abs(al - alpha_min) <= 1e-5:
            continue
        # termination-index difference: the extra ids form the tail of the longer list
        longer, shorter = (gpu, ora) if len(gpu) > len(ora) else (ora, gpu)
        if list(longer[: len(shorter)]) == list(shorter) or set(longer[: len(shorter)]) == set(shorter):
            T = 1.0
            for h in ora[: len(shorter)]:
                _, _, a = S.response(int(h), ro, rd)
                T *= 1.0 - min(a, 0.99)
            if abs(T - T_min) <= 1e-3 * T_min or abs(T - T_min) <= 2e-6:
                continue
        return False
    # same set, different order: every displaced pair must be a near tie in depth
    common_g = [g for g in gpu if g in so]
    common_o = [g for g in ora if g in sg]
    if common_g != common_o:
        for a_, b_ in zip(common_g, common_o):
            if a_ != b_:
                ta = S.response(int(a_), ro, rd)[0]
                tb = S.response(int(b_), ro, rd)[0]
                if abs(ta - tb) > 2e-6 * max(1.0, abs(ta)):
                    return False
    return True


def compare_hit_lists(S, rays, gpu_ids, gpu_nb, ora_ids, ora_nb, limit_report=5):
    """Indices of rays whose GPU and oracle blend lists differ in a way not excused."""
    o, d = rays[0], rays[1]
    bad = []
    for r in range(gpu_nb.shape[0]):
        a = [int(x) for x in gpu_ids[r, : gpu_nb[r]]]
        b = [int(x) for x in ora_ids[r, : ora_nb[r]]]
        if a == b:
            continue
        if not excused_mismatch(S, o[r], d[r], a, b):
            bad.append(r)
    return bad


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
