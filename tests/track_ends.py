"""Inputs with wires beyond the ends of the recorded track.

The refinement from the closest recorded state moves up to one recording interval along the track in
either direction (Sec. 2.2), so from the first or the last recorded state it reaches points beyond
the recorded track.  The wires built here cross the track's extension 0.875 of an interval past its
last recorded state and before its first one (and one between two interior states), perpendicular
to the track, at distance d0 from it: the closest recorded state is then ~14 mm from the wire while
the refined DCA is about d0.
"""
import numpy as np

import oracle as O


def end_case(field, S=40, stride=16, K=10, frac=0.875, d0=1e-3):
    """Returns (seeds [S][6], wires [6][3], hit_offsets, drift, n_steps); charge -1.  The seeds fan
    out in azimuth (2e-4 rad apart) from a 80 MeV/c, pz 30 MeV/c track at the origin; the track is
    recorded for K intervals of ``stride`` steps."""
    base = np.array([0.0, 0.0, 0.0, 80.0, 0.0, 30.0])
    seeds = []
    for i in range(S):
        a = (i - S // 2) * 2e-4
        pt = 80.0 * (1 + 1e-4 * (i % 7))
        seeds.append([0.0, 0.0, 0.0, pt * np.cos(a), pt * np.sin(a), 30.0])
    n_steps = stride * K
    ext = int(round(frac * stride))
    fine = O.Params(n_steps=n_steps + ext + 4, stride=1)
    fw, _ = O.propagate(field, fine, base[None], -1)
    bw, _ = O.propagate(field, fine, (base * [1, 1, 1, -1, -1, -1])[None], +1)   # time-reversed
    wires = []
    for st in (fw[0, n_steps + ext], bw[0, ext], fw[0, n_steps // 2 + ext // 2]):
        x, p = st[:3], st[3:]
        t = p / np.linalg.norm(p)
        n = np.cross(t, [0.0, 0.0, 1.0])
        n /= np.linalg.norm(n)
        u = np.cross(t, n)
        u /= np.linalg.norm(u)
        wires.append(np.r_[x + d0 * n, u])
    wires = np.ascontiguousarray(np.array(wires).T)
    return np.array(seeds), wires, np.arange(4, dtype=np.int32), np.full(3, d0), n_steps
