"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test fixes one part of the oracle against a closed form, an invariant, a special case that
reduces to textbook geometry, or brute force on a tiny input, so that a dropped term, a wrong sign, a
wrong index or a transposed operand anywhere in the oracle fails at least one of them:

* RK4 (Algorithm 1's extrapolator, fixed step): the closed-form helix in a uniform field, fourth-order
  convergence, |p| conservation in a pure magnetic field, exact straight lines at B = 0,
  time reversibility.
* DCA (Algorithm 2 / Sec. 2.2.2): line-line distance at B = 0, circle-point distance for axial wires,
  brute-force minimisation along the closed-form helix for stereo wires.
* RSS (Eq. 1): all-outlier and truth-seed special cases, and closed-form DCAs fed through the cap.
* Selection / classification (Sec. 2.1): brute force on tiny inputs.
* Determinism for any thread count (Sec. 4.1 requires it of the CPU computation).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1911_09340_gb300 import synth

KAPPA = synth.KAPPA
OPEN = dict(zmin=-50.0, zmax=50.0, rmax=50.0)   # target region that never stops the recording


def _helix_seed(vertex, p, pitch_deg, phi0):
    al = math.radians(pitch_deg)
    pt, pz = p * math.sin(al), p * math.cos(al)
    return np.array([*vertex, pt * math.cos(phi0), pt * math.sin(phi0), pz]), pt, pz


# ------------------------------------------------------------------------------------------------
# RK4
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("q,bz,pitch,p", [(-1, 1.0, 80.0, 104.0), (1, 1.0, 60.0, 90.0),
                                          (-1, 0.7, 87.0, 60.0), (-1, -1.0, 75.0, 104.97)])
def test_rk4_matches_closed_form_helix(q, bz, pitch, p):
    seed, pt, pz = _helix_seed((0.03, -0.02, -0.4), p, pitch, 0.3)
    P0 = math.hypot(pt, pz)
    turn = 2 * math.pi * P0 / (KAPPA * abs(bz))
    n = int(3 * turn / 1e-3)
    pts, nv = O.propagate(synth.uniform_field(bz), O.Params(n_steps=n, **OPEN), seed[None], q)
    assert nv[0] == n + 1
    s = np.arange(n + 1) * 1e-3
    pos, mom = synth.helix_points(seed[:3], pt, 0.3, pz, q, bz, s)
    assert np.abs(pts[0, :, :3] - pos.T).max() <= 1e-10
    assert np.abs(pts[0, :, 3:] - mom.T).max() <= 1e-10 * P0


def test_rk4_fourth_order():
    seed, pt, pz = _helix_seed((0.0, 0.0, 0.0), 104.0, 80.0, 0.0)
    P0 = math.hypot(pt, pz)
    L = 2 * math.pi * P0 / KAPPA          # one turn
    errs = []
    for h in (L / 128, L / 256, L / 512):
        n = int(round(L / h))
        pts, _ = O.propagate(synth.uniform_field(1.0), O.Params(h=h, n_steps=n, **OPEN), seed[None], -1)
        pos, _ = synth.helix_points(seed[:3], pt, 0.0, pz, -1, 1.0, np.array([n * h]))
        errs.append(np.abs(pts[0, -1, :3] - pos[:, 0]).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 14.0 <= r1 <= 18.0 and 14.0 <= r2 <= 18.0, (errs, r1, r2)


@pytest.mark.parametrize("kind", ["uniform", "table"])
def test_momentum_magnitude_conserved(kind):
    f = synth.uniform_field(1.0) if kind == "uniform" else synth.table_field(spacing=0.02)
    seed, pt, pz = _helix_seed((0.05, 0.01, -0.3), 103.0, 82.0, 1.1)
    P0 = math.hypot(pt, pz)
    pts, nv = O.propagate(f, O.Params(n_steps=6600, **OPEN), seed[None], -1)
    pmag = np.linalg.norm(pts[0, :nv[0], 3:], axis=1)
    assert np.abs(pmag / P0 - 1.0).max() <= 1e-12


def test_zero_field_is_a_straight_line():
    seed = np.array([0.1, -0.2, 0.3, 30.0, -40.0, 12.0])
    P0 = np.linalg.norm(seed[3:])
    pts, nv = O.propagate(synth.uniform_field(0.0), O.Params(n_steps=500, **OPEN), seed[None], -1)
    k = np.arange(nv[0])[:, None]
    expect = seed[:3] + k * 1e-3 * seed[3:] / P0
    assert np.abs(pts[0, :, :3] - expect).max() <= 1e-14
    assert np.abs(pts[0, :, 3:] - seed[3:]).max() == 0.0


def test_forward_then_backward_returns():
    f = synth.uniform_field(1.0)
    seed, pt, pz = _helix_seed((0.0, 0.05, 0.0), 104.0, 80.0, 2.0)
    P0 = math.hypot(pt, pz)
    y = seed.copy()
    for _ in range(2000):
        y = O.rk4_step(f, -1, P0, y, 1e-3)
    for _ in range(2000):
        y = O.rk4_step(f, -1, P0, y, -1e-3)
    assert np.abs(y[:3] - seed[:3]).max() <= 1e-10


def test_recording_stops_outside_target_region():
    seed = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 50.0])          # straight along +z at B = 0
    P = O.Params(n_steps=1000, stride=1, zmin=-1.0, zmax=0.1005, rmax=1.0)
    pts, nv = O.propagate(synth.uniform_field(0.0), P, seed[None], -1)
    # states at z = k mm; the first one beyond 0.1005 m is k = 101, recorded, then stop
    assert nv[0] == 102
    assert np.all(np.isnan(pts[0, nv[0]:]))
    P.stride = 4
    pts, nv = O.propagate(synth.uniform_field(0.0), P, seed[None], -1)
    assert nv[0] == 27     # recorded z = 0, 4, ..., 104 mm


def test_trilinear_exact_on_linear_field():
    # a trilinear interpolant reproduces any affine field exactly; a swapped axis or weight fails
    xs = -0.3 + 0.05 * np.arange(13)
    ys = -0.2 + 0.05 * np.arange(9)
    zs = -0.4 + 0.05 * np.arange(17)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    tab = np.stack([0.1 + 0.2 * X - 0.3 * Y + 0.4 * Z,
                    -0.5 + 0.6 * X + 0.7 * Y - 0.1 * Z,
                    1.0 - 0.2 * X + 0.05 * Y + 0.3 * Z]).astype(np.float32)
    # the float32 table holds these values only to ~6e-8; compare to the same rounding
    f = synth.Field(kind=1, table=tab, origin=(-0.3, -0.2, -0.4), spacing=0.05)
    rng = np.random.default_rng(5)
    for _ in range(50):
        x = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.2, 0.2), rng.uniform(-0.4, 0.4)])
        B = O.field_at(f, x)
        ex = [0.1 + 0.2 * x[0] - 0.3 * x[1] + 0.4 * x[2],
              -0.5 + 0.6 * x[0] + 0.7 * x[1] - 0.1 * x[2],
              1.0 - 0.2 * x[0] + 0.05 * x[1] + 0.3 * x[2]]
        assert np.allclose(B, ex, atol=3e-7, rtol=0)
    # outside the grid the coordinate is clamped to the edge
    B = O.field_at(f, np.array([5.0, -5.0, 0.0]))
    ex = [0.1 + 0.2 * 0.3 - 0.3 * -0.2, -0.5 + 0.6 * 0.3 + 0.7 * -0.2, 1.0 - 0.2 * 0.3 + 0.05 * -0.2]
    assert np.allclose(B, ex, atol=3e-7, rtol=0)


def test_constant_table_equals_uniform_field():
    tab = np.zeros((3, 5, 5, 5), np.float32)
    tab[2] = 1.0
    ft = synth.Field(kind=1, table=tab, origin=(-1.0, -1.0, -1.0), spacing=0.5)
    seed, _, _ = _helix_seed((0.02, 0.0, -0.3), 104.0, 80.0, 0.4)
    P = O.Params(n_steps=3000, **OPEN)
    a, _ = O.propagate(ft, P, seed[None], -1)
    b, _ = O.propagate(synth.uniform_field(1.0), P, seed[None], -1)
    assert np.abs(a - b).max() <= 1e-12


# ------------------------------------------------------------------------------------------------
# DCA
# ------------------------------------------------------------------------------------------------

def _scan_dca(field, seed, q, wires_aos, params, drift=None):
    W = wires_aos.shape[0]
    offs = np.arange(W + 1, dtype=np.int32)
    drift = np.zeros(W) if drift is None else drift
    r = O.scan(field, params, seed[None], q, wires_aos, offs, drift, np.zeros(W, np.uint8),
               want_dca=True, nthreads=1)
    return r


def test_dca_zero_field_is_line_line_distance():
    rng = np.random.default_rng(11)
    seed = np.array([0.0, 0.0, -0.3, 60.0, 20.0, 15.0])
    t = seed[3:] / np.linalg.norm(seed[3:])
    wires = []
    while len(wires) < 40:
        a = rng.uniform(-0.3, 0.6, 3)
        a[2] = 0.0
        u = rng.normal(size=3)
        u[2] = abs(u[2]) + 2.0
        u /= np.linalg.norm(u)
        # keep wires whose closest approach lies inside the recorded track (the method searches
        # near the closest recorded state)
        g = a - seed[:3]
        tu = t @ u
        ts = (g @ t - (g @ u) * tu) / (1.0 - tu * tu)
        if 0.05 < ts < 1.15:
            wires.append(np.concatenate([a, u]))
    wires = np.array(wires)
    r = _scan_dca(synth.uniform_field(0.0), seed, -1, wires, O.Params(n_steps=1200, **OPEN))
    for i, w in enumerate(wires):
        c = np.cross(t, w[3:])
        expect = abs(np.dot(w[:3] - seed[:3], c)) / np.linalg.norm(c)
        assert abs(r["dca"][0, i] - expect) <= 1e-12, (i, r["dca"][0, i], expect)
    assert r["n_unconv"][0] == 0


def test_dca_axial_wire_is_circle_distance():
    seed, pt, pz = _helix_seed((0.03, 0.0, -0.2), 104.0, 80.0, 0.3)
    q, bz = -1, 1.0
    R = pt / (KAPPA * bz)
    # centre of the transverse circle = the phase-independent part of the closed-form helix
    # x(s) = x0 - (pt/P0)(sin th - sin phi0)/w,  y(s) = y0 + (pt/P0)(cos th - cos phi0)/w
    P0 = math.hypot(pt, pz)
    w = KAPPA * q * bz / P0
    cx = seed[0] + (pt / P0) * math.sin(0.3) / w
    cy = seed[1] - (pt / P0) * math.cos(0.3) / w
    rng = np.random.default_rng(3)
    wires = []
    for _ in range(30):
        ang = rng.uniform(0, 2 * np.pi)
        rad = R + rng.uniform(-0.02, 0.02)
        wires.append([cx + rad * math.cos(ang), cy + rad * math.sin(ang), 0.0, 0.0, 0.0, 1.0])
    wires = np.array(wires)
    n = int(1.05 * 2 * math.pi * math.hypot(pt, pz) / KAPPA / 1e-3)
    r = _scan_dca(synth.uniform_field(bz), seed, q, wires, O.Params(n_steps=n, **OPEN))
    for i, wv in enumerate(wires):
        expect = abs(math.hypot(wv[0] - cx, wv[1] - cy) - R)
        assert abs(r["dca"][0, i] - expect) <= 1e-9, (i, r["dca"][0, i], expect)


def _brute_dca(seed, pt, pz, phi0, q, bz, wire, s_max):
    s = np.arange(0.0, s_max, 1e-4)
    pos, _ = synth.helix_points(seed[:3], pt, phi0, pz, q, bz, s)
    d = pos - wire[:3, None]
    t = (d * wire[3:, None]).sum(0)
    perp = np.linalg.norm(d - t * wire[3:, None], axis=0)
    k = int(np.argmin(perp))
    lo, hi = s[max(k - 1, 0)], s[min(k + 1, len(s) - 1)]
    g = (math.sqrt(5) - 1) / 2

    def f(sv):
        p_, _ = synth.helix_points(seed[:3], pt, phi0, pz, q, bz, np.array([sv]))
        dd = p_[:, 0] - wire[:3]
        tt = dd @ wire[3:]
        return np.linalg.norm(dd - tt * wire[3:])
    a, b = lo, hi
    for _ in range(80):
        c = b - g * (b - a)
        e = a + g * (b - a)
        if f(c) < f(e):
            b = e
        else:
            a = c
    return f(0.5 * (a + b))


def test_dca_stereo_wires_match_brute_force(chamber):
    ev = synth.make_event_fixed(chamber, np.random.default_rng(0), n_turns=1, sigma=0.0)
    seed = np.array([*ev.vertex, ev.pt * math.cos(ev.phi0), ev.pt * math.sin(ev.phi0), ev.pz])
    wires = O.wires_aos(ev.wires)[:12]
    n = ev.n_steps[0]
    r = _scan_dca(synth.uniform_field(1.0), seed, -1, wires, O.Params(n_steps=n, **OPEN))
    for i in range(wires.shape[0]):
        bf = _brute_dca(seed, ev.pt, ev.pz, ev.phi0, -1, 1.0, wires[i], n * 1e-3)
        assert abs(r["dca"][0, i] - bf) <= 1e-9, (i, r["dca"][0, i], bf)


def test_dca_same_for_every_recording_stride(chamber):
    ev = synth.single_event_fp64(chamber)
    seeds = O.lattice(ev.partitions[0])[::97]
    wires = O.wires_aos(ev.wires)
    mask = np.zeros(ev.n_hits, np.uint8)
    out = []
    for stride in (1, 3, 8, 16, 24, 32):
        P = O.Params(n_steps=ev.n_steps[0], stride=stride)
        out.append(O.scan(synth.uniform_field(1.0), P, seeds, -1, wires, ev.hit_offsets, ev.drift,
                          mask, want_dca=True))
    for o in out[1:]:
        near = out[0]["dca"] < 0.03          # same local minimum away from multi-pass ties
        assert np.abs(o["dca"][near] - out[0]["dca"][near]).max() <= 1e-9
        assert np.allclose(o["rss"], out[0]["rss"], rtol=1e-9, atol=1e-16)


# ------------------------------------------------------------------------------------------------
# RSS (Eq. 1)
# ------------------------------------------------------------------------------------------------

def _straight_setup():
    """B = 0 track along (cos 0.2, sin 0.2, 0) through the origin; axial wires at known offsets, so
    the DCA of wire i is exactly |offset_i|."""
    th = 0.2
    t = np.array([math.cos(th), math.sin(th), 0.0])
    nrm = np.array([-math.sin(th), math.cos(th), 0.0])
    offs = np.array([0.001, -0.004, 0.0025, 0.03, -0.0005, 0.012])
    along = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.6])
    wires = np.array([np.concatenate([al * t + o * nrm, [0, 0, 1.0]]) for al, o in zip(along, offs)])
    seed = np.array([0.0, 0.0, 0.0, *(50.0 * t)])
    return seed, wires, np.abs(offs)


def test_rss_closed_form_straight_track():
    seed, wires, D = _straight_setup()
    lam = 0.01
    # hits per wire: (drifts), some masked
    hits = [[0.0012], [0.0031, 0.0042, 0.0001], [0.0025], [0.0070], [0.0040, 0.0003], [0.0]]
    masked = [[0], [0, 0, 1], [0], [0], [1, 0], [1]]
    offs = np.cumsum([0] + [len(h) for h in hits]).astype(np.int32)
    drift = np.concatenate(hits)
    mask = np.concatenate(masked).astype(np.uint8)
    P = O.Params(n_steps=800, lam=lam, **OPEN)
    r = O.scan(synth.uniform_field(0.0), P, seed[None], -1, wires, offs, drift, mask, want_dca=True)
    assert np.allclose(r["dca"][0], D, atol=1e-13, rtol=0)
    # Eq. 1 by hand with the closed-form DCAs:
    #  w0: |0.001-0.0012| = 0.0002            -> 0.0002
    #  w1: D=0.004, unmasked 0.0031, 0.0042    -> min(0.0009, 0.0002) = 0.0002
    #  w2: D=0.0025, r=0.0025                  -> 0
    #  w3: D=0.03, r=0.007                     -> 0.023 capped at 0.01
    #  w4: D=0.0005, unmasked 0.0003           -> 0.0002
    #  w5: only hit masked                     -> wire absent from the sum
    expect = 0.0002 ** 2 + 0.0002 ** 2 + 0.0 + 0.01 ** 2 + 0.0002 ** 2
    assert abs(r["rss"][0] - expect) <= 1e-15
    assert r["n_in"][0] == 4


def test_rss_all_outliers_is_n_lambda_squared(chamber):
    ev = synth.single_event_fp64(chamber)
    seeds = O.lattice(ev.partitions[0])[::301]
    lam = 0.005
    drift = np.full(ev.n_hits, 5.0)        # 5 m: every residual exceeds the cutoff
    P = O.Params(n_steps=ev.n_steps[0], lam=lam)
    r = O.scan(synth.uniform_field(1.0), P, seeds, -1, O.wires_aos(ev.wires), ev.hit_offsets,
               drift, np.zeros(ev.n_hits, np.uint8))
    # N*lambda^2 up to the rounding of N sequential additions
    assert np.allclose(r["rss"], ev.n_wires * lam * lam, rtol=ev.n_wires * 2.3e-16, atol=0)
    assert np.all(r["n_in"] == 0)


def test_rss_truth_seed_on_noise_free_hits_is_zero(chamber):
    ev = synth.make_event_fixed(chamber, np.random.default_rng(1), n_turns=1, sigma=0.0)
    seed = np.array([*ev.vertex, ev.pt * math.cos(ev.phi0), ev.pt * math.sin(ev.phi0), ev.pz])
    P = O.Params(n_steps=ev.n_steps[0])
    r = O.scan(synth.uniform_field(1.0), P, seed[None], -1, O.wires_aos(ev.wires), ev.hit_offsets,
               ev.drift, np.zeros(ev.n_hits, np.uint8), want_dca=True)
    assert r["rss"][0] <= ev.n_wires * (1e-8) ** 2
    assert r["n_in"][0] == ev.n_wires


def test_empty_wire_list_gives_zero_rss():
    seed = np.array([0.0, 0.0, 0.0, 100.0, 0.0, 10.0])
    P = O.Params(n_steps=100, **OPEN)
    r = O.scan(synth.uniform_field(1.0), P, seed[None], -1, np.zeros((0, 6)), np.zeros(1, np.int32),
               np.zeros(0), np.zeros(0, np.uint8))
    assert r["rss"][0] == 0.0 and r["n_in"][0] == 0


def test_scan_is_deterministic_for_any_thread_count(chamber):
    ev = synth.single_event_fp64(chamber)
    seeds = O.lattice(ev.partitions[0])[::7]
    P = O.Params(n_steps=ev.n_steps[0])
    args = (synth.uniform_field(1.0), P, seeds, -1, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift,
            np.zeros(ev.n_hits, np.uint8))
    a = O.scan(*args, nthreads=1)
    b = O.scan(*args, nthreads=5)
    assert np.array_equal(a["rss"], b["rss"]) and np.array_equal(a["n_in"], b["n_in"])


# ------------------------------------------------------------------------------------------------
# Lattice, selection, classification
# ------------------------------------------------------------------------------------------------

def _blocked_expectation(spec):
    """Seeds in the blocked enumeration, built independently with meshgrid + reshape/transpose."""
    n = spec.counts
    b = [2 if n[0] % 2 == 0 else 1]
    b += [4 if n[d] % 4 == 0 else (2 if n[d] % 2 == 0 else 1) for d in (1, 2)]
    b.append(1)
    axes = [np.linspace(c - h, c + h, k) for c, h, k in zip(spec.centre, spec.half_width, n)]
    grids = np.meshgrid(*axes, indexing="ij")
    shape = (n[0] // b[0], b[0], n[1] // b[1], b[1], n[2] // b[2], b[2], n[3] // b[3], b[3])
    Z, PH, PZ, PT = [g.reshape(shape).transpose(0, 2, 4, 6, 1, 3, 5, 7).ravel() for g in grids]
    return np.stack([np.full_like(Z, spec.vxy[0]), np.full_like(Z, spec.vxy[1]), Z, PT * np.cos(PH),
                     PT * np.sin(PH), PZ], axis=1)


@pytest.mark.parametrize("counts", [(3, 4, 2, 5), (4, 6, 2, 8), (2, 2, 3, 6), (5, 8, 12, 3),
                                    (16, 16, 32, 32)])
def test_lattice_matches_meshgrid(counts):
    spec = synth.LatticeSpec(vxy=(0.01, -0.02), centre=(-0.1, 0.7, 15.0, 100.0),
                             half_width=(0.02, 0.04, 3.0, 6.4), counts=counts)
    seeds = O.lattice(spec)
    assert np.allclose(seeds, _blocked_expectation(spec), rtol=1e-15, atol=1e-15)
    one = synth.LatticeSpec(vxy=(0, 0), centre=(0.1, 0.2, 3.0, 90.0), half_width=(1, 1, 1, 1),
                            counts=(1, 1, 1, 1))
    s1 = O.lattice(one)
    assert np.allclose(s1[0], [0, 0, 0.1, 90 * math.cos(0.2), 90 * math.sin(0.2), 3.0], rtol=1e-15)


def test_lattice_blocks_are_neighbours():
    spec = synth.LatticeSpec(vxy=(0, 0), centre=(0.0, 0.0, 10.0, 100.0),
                             half_width=(0.02, 0.04, 3.0, 6.4), counts=(16, 16, 32, 32))
    seeds = O.lattice(spec)
    # every run of 32 consecutive seeds spans 2 nodes of z0, 4 of phi and pz, one pt
    step = np.array([0.04 / 15, 0.08 / 15, 6.0 / 31, 12.8 / 31])
    for blk in (0, 1, 777, 8191):
        s = seeds[blk * 32:(blk + 1) * 32]
        pt = np.hypot(s[:, 3], s[:, 4])
        ph = np.arctan2(s[:, 4], s[:, 3])
        span = np.array([np.ptp(s[:, 2]), np.ptp(ph), np.ptp(s[:, 5]), np.ptp(pt)])
        assert np.allclose(span, step * np.array([1, 3, 3, 0]), rtol=1e-9, atol=1e-12)


def test_select_matches_brute_force():
    rng = np.random.default_rng(2)
    for S in (1, 2, 7, 100, 1000):
        v = rng.integers(0, 5, size=S).astype(np.float64) * 0.25    # many ties
        if S > 3:
            v[rng.integers(0, S, size=2)] = np.nan
        order = sorted(range(S), key=lambda i: (math.isnan(v[i]), 0.0 if math.isnan(v[i]) else v[i], i))
        for k in (1, 3, 16):
            idx, val = O.select(v, k)
            kk = min(k, S)
            assert list(idx) == order[:kk]
            assert np.array_equal(val, v[order[:kk]], equal_nan=True)


def test_classify_closed_form_straight_track():
    seed, wires, D = _straight_setup()
    lam = 0.001
    hits = [[0.0012, 0.0009], [0.0031, 0.0042, 0.0039], [0.0025], [0.0070], [0.0040, 0.0003], [0.0]]
    masked = [[0, 0], [0, 0, 1], [0], [0], [1, 0], [1]]
    offs = np.cumsum([0] + [len(h) for h in hits]).astype(np.int32)
    drift = np.concatenate(hits)
    mask = np.concatenate(masked).astype(np.uint8)
    P = O.Params(n_steps=800, lam=lam, **OPEN)
    cls, dw, m2 = O.classify(synth.uniform_field(0.0), P, seed, -1, wires, offs, drift, mask,
                             update_mask=True)
    # w0 D=0.001: e = 0.0002, 0.0001 -> second hit (tie-free) classified
    # w1 D=0.004: unmasked e = 0.0009, 0.0002 -> hit 1 classified; hit 2 masked
    # w2 D=0.0025: e = 0 -> classified
    # w3 D=0.03: e = 0.023 >= lam -> none
    # w4 D=0.0005: unmasked hit 1: e = 0.0002 -> classified
    # w5: only hit masked -> none
    expect = np.array([0, 1, 0, 1, 0, 1, 0, 0, 1, 0], np.uint8)
    assert np.array_equal(cls, expect)
    assert np.allclose(dw, D, atol=1e-13, rtol=0)
    assert np.array_equal(m2, mask | expect)


def test_classify_ties_take_the_lowest_hit_index():
    seed, wires, D = _straight_setup()
    wires = wires[:1]
    drift = np.array([0.0003, 0.0008, 0.0008])        # D = 0.001: hits 1 and 2 tie exactly
    offs = np.array([0, 3], np.int32)
    P = O.Params(n_steps=800, lam=0.01, **OPEN)
    cls, _, _ = O.classify(synth.uniform_field(0.0), P, seed, -1, wires, offs, drift,
                           np.zeros(3, np.uint8))
    assert np.array_equal(cls, np.array([0, 1, 0], np.uint8))


@pytest.mark.parametrize("stride", [1, 4, 16])
def test_refined_dca_stays_in_its_valley(chamber, stride):
    # the continuous distance minimum near the closest recorded state lies within half a recording
    # interval (in arc length) of a recorded state, so the refined DCA can be at most h_rec/2 below
    # the closest recorded distance; the refined state stays within one interval of that state, so
    # at most h_rec above it; and near wires (where the refinement converges) end below it
    ev = synth.multi_turn_event(0, chamber)
    seeds = O.lattice(ev.partitions[0])[::4099]
    P = O.Params(n_steps=ev.n_steps[0], stride=stride)
    wires = O.wires_aos(ev.wires)
    r = O.scan(synth.uniform_field(1.0), P, seeds, -1, wires, ev.hit_offsets, ev.drift,
               np.zeros(ev.n_hits, np.uint8), want_dca=True)
    pts, nv = O.propagate(synth.uniform_field(1.0), P, seeds, -1)
    h_rec = 1e-3 * stride
    for s in range(seeds.shape[0]):
        x = pts[s, :nv[s], :3]
        for i, w in enumerate(wires):
            d = x - w[:3]
            t = d @ w[3:]
            dmin = np.linalg.norm(d - t[:, None] * w[3:], axis=1).min()
            D = r["dca"][s, i]
            assert dmin - 0.5 * h_rec - 1e-12 <= D <= dmin + h_rec + 1e-12
            if dmin < 0.05:
                assert D <= dmin + 1e-12


def test_backward_seed_retraces_the_turn():
    """Flipping q and p at the end of a turn (the exit-side half track, Sec. 3.1) retraces the turn:
    the backward recording, read in reverse, is the forward one; the backward lattice of
    synth.backward_partition is centred on that reversed state with the forward lattice's offsets."""
    ev = synth.single_event_fp64()
    field = synth.uniform_field(1.0)
    n = int(ev.s_turn / 1e-3)
    tr0 = np.array([*ev.vertex, ev.pt * math.cos(ev.phi0), ev.pt * math.sin(ev.phi0), ev.pz])
    P = O.Params(n_steps=n, stride=1, **OPEN)
    fwd, _ = O.propagate(field, P, tr0[None], ev.q)
    pos, mom = synth.helix_points(ev.vertex, ev.pt, ev.phi0, ev.pz, ev.q, 1.0, np.array([n * 1e-3]))
    end = np.array([*pos[:, 0], *(-mom[:, 0])])
    bwd, _ = O.propagate(field, P, end[None], -ev.q)
    assert np.abs(bwd[0, :, :3] - fwd[0, ::-1, :3]).max() <= 1e-9
    assert np.abs(bwd[0, :, 3:] + fwd[0, ::-1, 3:]).max() <= 1e-9 * ev.p
    spec, back = ev.partitions[0], synth.backward_partition(ev, 0)
    dz_turn = ev.pz / ev.p * ev.s_turn
    assert back.charge == -spec.charge and back.counts == spec.counts
    assert back.centre[0] - spec.centre[0] == pytest.approx(dz_turn, abs=1e-12)
    assert math.cos(back.centre[1] - spec.centre[1]) == pytest.approx(-1.0, abs=1e-12)
    assert back.centre[2] == -spec.centre[2] and back.centre[3] == spec.centre[3]


def test_refinement_reaches_beyond_the_recorded_track():
    """A wire crossing the track 0.875 of an interval past its last recorded state (or before its
    first): the oracle's DCA equals the brute-force minimum of the distance over the track propagated
    in 10 um steps (the refinement moves up to one interval from the closest recorded state)."""
    from track_ends import end_case
    U = synth.uniform_field(1.0)
    seeds, wires, offs, drift, n = end_case(U, S=3)
    P = O.Params(n_steps=n, stride=16, lam=2e-3, tol=1e-12)
    wa = O.wires_aos(wires)
    r = O.scan(U, P, seeds, -1, wa, offs, drift, np.zeros(3, np.uint8), want_dca=True)
    fine = O.Params(h=1e-5, n_steps=200 * 100, stride=1)
    for s in range(3):
        for back in (False, True):
            sd = seeds[s] * ([1, 1, 1, -1, -1, -1] if back else 1)
            pts, nv = O.propagate(U, fine, sd[None], 1 if back else -1)
            i = 1 if back else 0
            lo = 150 * 100 if not back else 0
            x = pts[0, lo: lo + 40 * 100, :3]
            d = x - wa[i, :3]
            d = d - (d @ wa[i, 3:])[:, None] * wa[i, 3:]
            brute = np.sqrt((d * d).sum(1)).min()
            assert abs(r["dca"][s, i] - brute) <= 1e-7, (s, i, r["dca"][s, i], brute)
            assert brute < 1.5e-3


def _golden(name):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if len(line) == 2:
                vals[line[0]] = float(line[1])
    return vals


def test_helix_radius_and_pitch_follow_eq3():
    """The recorded track of a 104.97 MeV/c electron with p_T = 101 MeV/c in 1 T (tests/golden/
    helix_curvature.txt, Eq. 3): the circle through its transverse positions has radius
    p_T / (0.3 B) mm to the rounding of Eq. 3's 0.3 (7e-4 relative), p_T / (kappa B) to 1e-9 m with
    the exact kappa, and the track advances 2 pi R p_z / p_T along z per turn."""
    g = _golden("helix_curvature.txt")
    pT, p, B = g["pT_MeV"], g["p_MeV"], g["B_T"]
    pz = math.sqrt(p * p - pT * pT)
    R_eq3 = pT / (g["kappa_eq3"] * B) * 1e-3          # m
    R_exact = pT / (299.792458 * B)
    n = 2200
    seed = np.array([[0.0, 0.0, 0.0, pT, 0.0, pz]])
    pts, nv = O.propagate(synth.uniform_field(B), O.Params(n_steps=n, **OPEN), seed, -1)
    x, y, z = pts[0, : nv[0], 0], pts[0, : nv[0], 1], pts[0, : nv[0], 2]
    # algebraic circle fit x^2 + y^2 + D x + E y + F = 0 (least squares)
    A = np.stack([x, y, np.ones_like(x)], axis=1)
    D, E, F = np.linalg.lstsq(A, -(x * x + y * y), rcond=None)[0]
    R = math.sqrt(D * D / 4 + E * E / 4 - F)
    assert abs(R - R_eq3) / R_eq3 < 1e-3
    assert abs(R - R_exact) < 1e-9
    # z advance per turn: z(s) = (p_z / p) s, one turn is s = 2 pi R p / p_T
    s_turn = 2 * math.pi * R_exact * p / pT
    k = int(round(s_turn / 1e-3))
    assert abs(z[k] - pz / p * k * 1e-3) < 1e-12
    assert abs(math.hypot(x[k], y[k])) < 2e-3           # back near the start after one turn
