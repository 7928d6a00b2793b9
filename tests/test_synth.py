"""The seeded input generator: reproducible, and its simulated hits agree with closed-form geometry."""
import math

import numpy as np

from paper_1911_09340_gb300 import synth


def test_chamber_geometry(chamber):
    assert chamber.n_wires == 18 * 300
    assert np.allclose(np.linalg.norm(chamber.u, axis=0), 1.0)
    assert np.isclose(chamber.radii[0], 0.50) and np.isclose(chamber.radii[-1], 0.84)
    # stereo angle alternates +-4 deg with the layer
    ang = np.degrees(np.arccos(chamber.u[2]))
    assert np.allclose(ang, 4.0)
    tphi = np.stack([-np.sin(chamber.phi), np.cos(chamber.phi), np.zeros_like(chamber.phi)])
    sgn = np.sign((chamber.u * tphi).sum(0))
    assert np.all(sgn == np.where(chamber.layer % 2 == 0, 1, -1))


def test_events_are_reproducible(chamber):
    a = synth.multi_turn_event(3, chamber)
    b = synth.multi_turn_event(3, chamber)
    assert np.array_equal(a.drift, b.drift) and np.array_equal(a.wire_ids, b.wire_ids)
    assert a.partitions == b.partitions


def test_axial_chamber_hits_match_circle_distance():
    ch = synth.make_chamber(stereo_deg=0.0)
    ev = synth.make_event_fixed(ch, np.random.default_rng(0), n_turns=1, sigma=0.0)
    P0 = math.hypot(ev.pt, ev.pz)
    w = synth.KAPPA * ev.q * 1.0 / P0
    cx = ev.vertex[0] + (ev.pt / P0) * math.sin(ev.phi0) / w
    cy = ev.vertex[1] - (ev.pt / P0) * math.cos(ev.phi0) / w
    R = ev.pt / synth.KAPPA
    wid = np.repeat(np.arange(ev.n_wires), np.diff(ev.hit_offsets))
    a = ev.wires[:3, wid]
    expect = np.abs(np.hypot(a[0] - cx, a[1] - cy) - R)
    assert np.abs(ev.hit_dtrue - expect).max() < 1e-9
    # every wire within 8 mm of the circle in the layers the track crosses fired
    rho_max = math.hypot(cx, cy) + R
    d_all = np.abs(np.hypot(ch.a[0] - cx, ch.a[1] - cy) - R)
    # wires whose circle point lies on the one-turn track (all of the circle) and inside the chamber
    want = set(np.nonzero(d_all < 8e-3 - 1e-6)[0]) - set(np.nonzero(np.abs(d_all - 8e-3) < 1e-6)[0])
    assert want == set(ev.wire_ids.tolist()) or rho_max < ch.radii[0]


def test_window_on_fired_wires(chamber):
    for i in range(5):
        ev = synth.multi_turn_event(i, chamber)
        fired = np.unique(np.repeat(ev.wire_ids, np.diff(ev.hit_offsets))[ev.hit_turn >= 0])
        assert 60 <= fired.size <= 250
        assert 2 <= ev.n_turns <= 5
        n_sig = int((ev.hit_turn >= 0).sum())
        assert int((ev.hit_turn < 0).sum()) == round(0.1 * n_sig)
        assert len(ev.partitions) == ev.n_turns and ev.partitions[0].n_seeds == 2 ** 18
