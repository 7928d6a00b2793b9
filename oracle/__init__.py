"""FP64 CPU oracle of the seed scan -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import this package.  The CUDA library never calls it and shares no code with it; ``oracle.c``
states, function by function, which part of the paper it follows (Eq. 1, Algorithms 1-3, Sec. 2.1
and Sec. 2.2).

Arrays crossing into C are float64 / int32 / int8 / uint8, C-contiguous, in the oracle's own AoS
layouts (seeds [S][6], points [S][n_rec][6], wires [W][6]); the helpers below convert from the
generator's [6][W] wire layout.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, so x86 and Arm give identical results)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("b", C.c_double * 3), ("table", C.c_void_p),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("origin", C.c_double * 3), ("spacing", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("h", C.c_double), ("n_steps", C.c_int), ("stride", C.c_int),
                ("lam", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int),
                ("zmin", C.c_double), ("zmax", C.c_double), ("rmax", C.c_double)]


@dataclass
class Params:
    """Scan parameters (see ``or_params`` in oracle.c)."""
    h: float = 1e-3
    n_steps: int = 2200
    stride: int = 1
    lam: float = 1e-2
    tol: float = 1e-12
    max_iter: int = 16
    zmin: float = -0.80
    zmax: float = 0.80
    rmax: float = 0.90

    def n_rec(self) -> int:
        return self.n_steps // self.stride + 1

    def _c(self) -> _Params:
        return _Params(self.h, self.n_steps, self.stride, self.lam, self.tol, self.max_iter,
                       self.zmin, self.zmax, self.rmax)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            vp = C.c_void_p
            lib.oracle_lattice.argtypes = [C.c_double, C.c_double, vp, vp, vp, vp]
            lib.oracle_propagate.argtypes = [P(_Field), P(_Params), vp, vp, C.c_int64, vp, vp,
                                             C.c_int]
            lib.oracle_scan.argtypes = [P(_Field), P(_Params), vp, vp, C.c_int64, vp, C.c_int,
                                        vp, vp, vp, vp, vp, vp, vp, C.c_int]
            lib.oracle_select.argtypes = [vp, C.c_int64, C.c_int, vp, vp]
            lib.oracle_classify.argtypes = [P(_Field), P(_Params), vp, C.c_int, vp, C.c_int, vp,
                                            vp, vp, vp, vp, C.c_int]
            lib.oracle_rk4_step.argtypes = [P(_Field), C.c_int, C.c_double, vp, C.c_double]
            lib.oracle_field_at.argtypes = [P(_Field), vp, vp]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class FieldC:
    """Keeps the C field struct and the table it points to alive together."""

    def __init__(self, field):
        self.table = None
        if field.kind == 0:
            self.c = _Field(0, (C.c_double * 3)(*field.b), None, 0, 0, 0,
                            (C.c_double * 3)(0, 0, 0), 0.0)
        else:
            self.table = np.ascontiguousarray(field.table, dtype=np.float32)
            nz, ny, nx = self.table.shape[1:]
            self.c = _Field(1, (C.c_double * 3)(*field.b), self.table.ctypes.data, nx, ny, nz,
                            (C.c_double * 3)(*field.origin), float(field.spacing))


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def lattice(spec) -> np.ndarray:
    """Seeds [S][6] of a ``synth.LatticeSpec``."""
    seeds = np.empty((spec.n_seeds, 6), np.float64)
    cen = _f64(spec.centre)
    hw = _f64(spec.half_width)
    cnt = np.ascontiguousarray(spec.counts, dtype=np.int32)
    _load().oracle_lattice(float(spec.vxy[0]), float(spec.vxy[1]), _ptr(cen), _ptr(hw), _ptr(cnt),
                           _ptr(seeds))
    return seeds


def propagate(field, params: Params, seeds, charge, nthreads=None):
    """Returns (points [S][n_rec][6], n_valid [S])."""
    seeds = _f64(seeds)
    S = seeds.shape[0]
    charge = np.ascontiguousarray(np.broadcast_to(charge, (S,)), dtype=np.int8)
    pts = np.full((S, params.n_rec(), 6), np.nan)
    nv = np.zeros(S, np.int32)
    fc = FieldC(field)
    _load().oracle_propagate(C.byref(fc.c), C.byref(params._c()), _ptr(seeds), _ptr(charge), S,
                             _ptr(pts), _ptr(nv), nthreads or default_threads())
    return pts, nv


def wires_aos(wires_soa) -> np.ndarray:
    """[6][W] -> [W][6]."""
    return np.ascontiguousarray(np.asarray(wires_soa, dtype=np.float64).T)


def scan(field, params: Params, seeds, charge, wires, hit_offsets, drift, mask,
         want_dca=False, nthreads=None):
    """RSS of every seed.  ``wires`` is [W][6].  Returns dict(rss, n_in, n_unconv[, dca [S][W]])."""
    seeds = _f64(seeds)
    S = seeds.shape[0]
    charge = np.ascontiguousarray(np.broadcast_to(charge, (S,)), dtype=np.int8)
    wires = _f64(wires)
    W = wires.shape[0]
    offs = np.ascontiguousarray(hit_offsets, dtype=np.int32)
    drift = _f64(drift)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    rss = np.zeros(S)
    n_in = np.zeros(S, np.int32)
    nunc = np.zeros(S, np.int32)
    dca = np.full((S, W), np.nan) if want_dca else None
    fc = FieldC(field)
    _load().oracle_scan(C.byref(fc.c), C.byref(params._c()), _ptr(seeds), _ptr(charge), S,
                        _ptr(wires), W, _ptr(offs), _ptr(drift), _ptr(mask), _ptr(rss), _ptr(n_in),
                        _ptr(dca), _ptr(nunc), nthreads or default_threads())
    out = dict(rss=rss, n_in=n_in, n_unconv=nunc)
    if want_dca:
        out["dca"] = dca
    return out


def select(rss, k=1):
    """(idx [k] int64, rss [k]) of the k lowest RSS, ties by lowest index, NaN last."""
    rss = _f64(rss)
    k = min(k, rss.shape[0])
    idx = np.zeros(k, np.int64)
    val = np.zeros(k)
    _load().oracle_select(_ptr(rss), rss.shape[0], k, _ptr(idx), _ptr(val))
    return idx, val


def classify(field, params: Params, seed, q, wires, hit_offsets, drift, mask, update_mask=False):
    """Returns (hit_class [H] uint8, dca_wire [W], mask_after [H])."""
    seed = _f64(seed).reshape(6)
    wires = _f64(wires)
    W = wires.shape[0]
    offs = np.ascontiguousarray(hit_offsets, dtype=np.int32)
    drift = _f64(drift)
    m = np.array(mask, dtype=np.uint8, copy=True)
    H = int(offs[-1])
    cls = np.zeros(H, np.uint8)
    dw = np.full(W, np.nan)
    fc = FieldC(field)
    _load().oracle_classify(C.byref(fc.c), C.byref(params._c()), _ptr(seed), int(q), _ptr(wires), W,
                            _ptr(offs), _ptr(drift), _ptr(m), _ptr(cls), _ptr(dw), int(update_mask))
    return cls, dw, m


def rk4_step(field, q, P0, y, h):
    y = _f64(y).copy()
    fc = FieldC(field)
    _load().oracle_rk4_step(C.byref(fc.c), int(q), float(P0), _ptr(y), float(h))
    return y


def field_at(field, x):
    x = _f64(x)
    B = np.zeros(3)
    fc = FieldC(field)
    _load().oracle_field_at(C.byref(fc.c), _ptr(x), _ptr(B))
    return B


def scan_partition(field, params: Params, spec, wires, hit_offsets, drift, mask, k=1,
                   want_dca=False, nthreads=None, update_mask=True):
    """One turn partition end to end: lattice -> RSS -> select -> classify (+ mask update)."""
    seeds = lattice(spec)
    res = scan(field, params, seeds, spec.charge, wires, hit_offsets, drift, mask, want_dca,
               nthreads)
    idx, val = select(res["rss"], k)
    cls, dw, m2 = classify(field, params, seeds[idx[0]], spec.charge, wires, hit_offsets, drift,
                           mask, update_mask)
    res.update(seeds=seeds, idx=idx, best_rss=val, hit_class=cls, dca_wire=dw, mask=m2)
    return res


def refine_refs(seeds, idx, half_width, K):
    """Sec. 2.1, iterative refinement: "several seeds with the lowest RSS are selected as reference
    points for the next seed scanning", kept "sparse enough to avoid overlaps between new seed sets".
    Walks the candidate indices in the given order (ascending RSS) and keeps a candidate unless an
    already kept reference lies closer than 2 * half_width[d] in every lattice coordinate d of
    (z0, phi, pz, pT) (phi modulo 2 pi), i.e. unless the two new lattices would overlap; stops at K.
    ``seeds`` is AoS [S][6].  Returns the kept references as an [n, 4] float64 array."""
    seeds = np.asarray(seeds, dtype=np.float64)
    hw = np.asarray(half_width, dtype=np.float64)
    kept = []
    for s in np.asarray(idx).tolist():
        if len(kept) == K:
            break
        if s < 0 or s >= seeds.shape[0]:
            continue
        x = seeds[s]
        c = np.array([x[2], np.arctan2(x[4], x[3]), x[5], np.hypot(x[3], x[4])])
        clash = False
        for r in kept:
            d = c - r
            d[1] = np.remainder(d[1] + np.pi, 2.0 * np.pi) - np.pi
            if np.all(np.abs(d) < 2.0 * hw):
                clash = True
                break
        if not clash:
            kept.append(c)
    return np.array(kept, dtype=np.float64).reshape(-1, 4)


def lattice_refined(shape, refs, K):
    """The finer scan's seeds: K lattices of ``shape``'s vertex, half-widths and counts, lattice k
    centred at refs[k] (refs[0] again for k beyond the references found), one after the other, each
    in the oracle's lattice order.  Returns AoS [K * S1][6]."""
    import dataclasses as _dc
    refs = np.asarray(refs, dtype=np.float64).reshape(-1, 4)
    out = []
    for k in range(K):
        c = refs[k] if k < refs.shape[0] else refs[0]
        out.append(lattice(_dc.replace(shape, centre=tuple(float(v) for v in c))))
    return np.concatenate(out, axis=0)


def seeds_from_theta(theta, vx, vy):
    """Seeds (AoS [S][6]) of lattice coordinates theta [S][4] = (z0, phi, pz, pT) at vertex (vx, vy),
    as the lattice builds them (Sec. 2.1)."""
    th = np.asarray(theta, dtype=np.float64).reshape(-1, 4)
    n = th.shape[0]
    return np.stack([np.full(n, vx), np.full(n, vy), th[:, 0], th[:, 3] * np.cos(th[:, 1]),
                     th[:, 3] * np.sin(th[:, 1]), th[:, 2]], axis=1)


def smoothed_rss(field, params: Params, theta, vx, vy, q, wires, hit_offsets, drift, mask, tau):
    """Eq. 1 with a smooth cap, for Gauss-Newton refinement of the best seeds: for every wire with an
    unmasked hit, e = min_j |D - r_j| (D from this oracle's scan), w = 1 / (1 + exp(-(lam - e)/tau)),
    term = w e^2 + (1 - w) lam^2; summed in ascending wire order.  Returns (srss [S], dca [S][W])."""
    return smoothed_rss_seeds(field, params, seeds_from_theta(theta, vx, vy), q, wires, hit_offsets,
                              drift, mask, tau)


def smoothed_rss_seeds(field, params: Params, seeds, q, wires, hit_offsets, drift, mask, tau):
    """smoothed_rss of Cartesian seeds (AoS [S][6])."""
    seeds = np.asarray(seeds, dtype=np.float64).reshape(-1, 6)
    r = scan(field, params, seeds, q, wires, hit_offsets, drift, mask, want_dca=True)
    D = r["dca"]
    offs = np.asarray(hit_offsets)
    dr = np.asarray(drift, dtype=np.float64)
    mk = np.asarray(mask)
    lam = params.lam
    out = np.zeros(seeds.shape[0])
    for s in range(seeds.shape[0]):
        tot = 0.0
        for i in range(offs.shape[0] - 1):
            live = [j for j in range(offs[i], offs[i + 1]) if not mk[j]]
            if not live:
                continue
            e = min(abs(D[s, i] - dr[j]) for j in live)
            x = (lam - e) / tau
            w = 1.0 / (1.0 + np.exp(-x)) if x >= 0 else np.exp(x) / (1.0 + np.exp(x))
            tot += w * e * e + (1.0 - w) * lam * lam
        out[s] = tot
    return out, D
