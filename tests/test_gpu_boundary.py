"""Argument validation at the C ABI (include/comet_scan.h): every entry point, given one invalid
argument at a time, returns COMET_ERR_INVALID_ARG before launching anything -- its output arrays keep
the sentinel they were filled with, and the CUDA context has no pending error.  Called through ctypes
directly (no binding-side checks in the way); every other argument is a valid device array.  No
call in this file reaches a kernel launch."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1911_09340_gb300 import binding as B
from paper_1911_09340_gb300 import synth

pytestmark = pytest.mark.gpu
INVALID = 1
S, NREC, W, H = 64, 9, 4, 6


def _p(t):
    return C.c_void_p(t.data_ptr())


def _odd(t):
    """A pointer one byte past t's start: misaligned for every element type."""
    return C.c_void_p(t.data_ptr() + 1)


def _params(**kw):
    base = dict(n_steps=8, stride=1, lam=0.01, tol=1e-6)
    base.update(kw)
    return B.ScanParams(**base).c()


def _field(kind=0, table=None):
    f = B.DeviceField(kind=0, b=(0.0, 0.0, 1.0)).c()
    f.kind = kind
    if table is not None:
        f.table = table
    return f


@pytest.fixture(scope="module")
def bufs():
    d = "cuda"
    spec = synth.LatticeSpec(vxy=(0.0, 0.0), centre=(0.0, 0.3, 20.0, 100.0),
                             half_width=(0.01, 0.02, 1.0, 2.0), counts=(2, 2, 4, 4), charge=-1)
    b = dict(
        spec=spec,
        seeds=torch.zeros((6, S), dtype=torch.float32, device=d),
        charge=torch.full((S,), -1, dtype=torch.int8, device=d),
        points=torch.full((6, NREC, S), 7.0, dtype=torch.float32, device=d),
        n_valid=torch.full((S,), 7, dtype=torch.int32, device=d),
        bounds=torch.full(B.bounds_shape(S), 7.0, dtype=torch.float32, device=d),
        wires=torch.zeros((6, W), dtype=torch.float32, device=d),
        offs=torch.arange(0, 2 * W + 1, 2, dtype=torch.int32, device=d)[: W + 1].contiguous(),
        drift=torch.full((2 * W,), 1e-3, dtype=torch.float32, device=d),
        mask=torch.zeros(2 * W, dtype=torch.uint8, device=d),
        rss=torch.full((S,), 7.0, dtype=torch.float32, device=d),
        n_in=torch.full((S,), 7, dtype=torch.int32, device=d),
        idx=torch.full((64,), 7, dtype=torch.int64, device=d),
        val=torch.full((64,), 7.0, dtype=torch.float32, device=d),
        hit_class=torch.full((2 * W,), 7, dtype=torch.uint8, device=d),
        theta=torch.full((S, 4), 7.0, dtype=torch.float64, device=d),
        refs=torch.full((32, 4), 7.0, dtype=torch.float64, device=d),
        nrefs=torch.full((1,), 7, dtype=torch.int32, device=d),
    )
    b["wires"][5] = 1.0          # unit directions along z
    return b


def _untouched(b):
    torch.cuda.synchronize()
    for k in ("points", "n_valid", "bounds", "rss", "n_in", "idx", "val", "hit_class", "theta",
              "refs", "nrefs"):
        t = b[k]
        assert bool((t == 7).all()), k


def _expect_invalid(rc):
    assert rc == INVALID, (rc, B.lib().comet_last_error().decode())
    assert B.lib().comet_last_error().decode() != ""


def test_propagate_validation(ctx, bufs):
    L, b = B.lib(), bufs
    P = lambda **kw: C.byref(_params(**kw))
    F = C.byref(_field())
    st = None
    good = [ctx.handle, 0, F, P(), _p(b["seeds"]), _p(b["charge"]), S, _p(b["points"]), _p(b["n_valid"]),
            _p(b["bounds"]), st]
    bad = {
        0: [None], 1: [7, -1], 2: [None, C.byref(_field(kind=3)), C.byref(_field(kind=1, table=None))],
        3: [None, P(h=0.0), P(h=float("nan")), P(n_steps=0), P(stride=0), P(zmin=float("nan"))],
        4: [None, _odd(b["seeds"])], 5: [None], 6: [-1], 7: [None, _odd(b["points"])],
        8: [None, _odd(b["n_valid"])], 9: [C.c_void_p(b["bounds"].data_ptr() + 4)],
    }
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_propagate(*args))
    _untouched(b)


def test_dca_validation(ctx, bufs):
    L, b = B.lib(), bufs
    P = lambda **kw: C.byref(_params(**kw))
    good = [ctx.handle, 0, C.byref(_field()), P(), _p(b["points"]), _p(b["n_valid"]), _p(b["charge"]), S,
            None, _p(b["wires"]), W, W, _p(b["offs"]), _p(b["drift"]), _p(b["mask"]), _p(b["rss"]),
            _p(b["n_in"]), None, None, None, None, None]
    bad = {
        0: [None], 1: [2], 2: [None],
        3: [None, P(lam=0.0), P(lam=-1.0), P(tol=0.0), P(max_iter=-1), P(n_steps=0), P(stride=0)],
        4: [None, _odd(b["points"])], 5: [None], 6: [None], 7: [-5],
        8: [C.c_void_p(b["bounds"].data_ptr() + 8)],
        9: [None, _odd(b["wires"])], 10: [-1], 11: [W - 1], 12: [None, _odd(b["offs"])],
        13: [None, _odd(b["drift"])], 14: [None], 15: [None, _odd(b["rss"])], 16: [None, _odd(b["n_in"])],
        17: [_odd(b["rss"])], 18: [_odd(b["n_in"])], 19: [_odd(b["idx"])],
        20: [_odd(b["rss"]), _p(b["val"])],     # misaligned; an RSS output without the index output
    }
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_dca(*args))
    _untouched(b)


def test_select_and_noalloc_validation(ctx, bufs):
    L, b = B.lib(), bufs
    good = [ctx.handle, 0, _p(b["rss"]), S, 1, _p(b["idx"]), _p(b["val"]), None]
    bad = {0: [None], 1: [9], 2: [None, _odd(b["rss"])], 3: [0, -3], 4: [0, 65, S + 1],
           5: [None, _odd(b["idx"])], 6: [_odd(b["val"])]}
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_select(*args))
    host = np.zeros(S, np.float32)
    good = [0, _p(b["rss"]), S, 1, _p(b["idx"]), _p(b["val"]), None]
    bad = {0: [9], 1: [None, _odd(b["rss"]), C.c_void_p(host.ctypes.data)], 2: [0], 3: [0, 65],
           4: [None, _odd(b["idx"])], 5: [_odd(b["val"])]}
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_select_noalloc(*args))
    _untouched(b)


def test_classify_validation(ctx, bufs):
    L, b = B.lib(), bufs
    P = lambda **kw: C.byref(_params(**kw))
    si = torch.zeros(1, dtype=torch.int64, device="cuda")
    good = [ctx.handle, 0, C.byref(_field()), P(), _p(b["points"]), _p(b["n_valid"]), _p(b["charge"]), S,
            _p(si), _p(b["wires"]), W, W, _p(b["offs"]), _p(b["drift"]), _p(b["mask"]), _p(b["hit_class"]),
            None, 1, None]
    bad = {
        0: [None], 1: [3], 2: [None], 3: [None, P(lam=0.0), P(tol=-1.0), P(n_steps=0)],
        4: [None, _odd(b["points"])], 5: [None], 6: [None], 7: [0], 8: [None, _odd(si)],
        9: [None], 10: [-2], 11: [1], 12: [None], 13: [None], 14: [None], 15: [None],
        16: [_odd(b["val"])],
    }
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_classify(*args))
    _untouched(b)


def test_lattice_refine_jacobian_gn_validation(ctx, bufs):
    L, b = B.lib(), bufs
    lat = B.lattice_struct(b["spec"])
    badlat = B.lattice_struct(b["spec"])
    badlat.counts[2] = 0
    nanlat = B.lattice_struct(b["spec"])
    nanlat.centre[1] = float("nan")
    qlat = B.lattice_struct(b["spec"])
    qlat.charge = 300
    good = [ctx.handle, 0, C.byref(lat), _p(b["points"]), None, S, None]
    bad = {0: [None], 1: [4], 2: [None, C.byref(badlat), C.byref(nanlat), C.byref(qlat)],
           3: [None, _odd(b["points"])], 5: [S - 1, 0]}
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_lattice(*args))
    hw = (C.c_double * 4)(0.01, 0.01, 0.5, 0.5)
    neg = (C.c_double * 4)(0.01, -0.01, 0.5, 0.5)
    good = [ctx.handle, 0, _p(b["points"]), S, _p(b["idx"]), 8, hw, 4, _p(b["refs"]), _p(b["nrefs"]), None]
    bad = {0: [None], 2: [None], 3: [0], 4: [None, _odd(b["idx"])], 5: [0, (1 << 20) + 1], 6: [None, neg],
           7: [0, 33], 8: [None, _odd(b["refs"])], 9: [None, _odd(b["nrefs"])]}
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_refine_refs(*args))
    good = [ctx.handle, 0, C.byref(lat), _p(b["refs"]), _p(b["nrefs"]), 1, _p(b["points"]), None, S, None]
    bad = {0: [None], 2: [None, C.byref(badlat)], 3: [None], 4: [None], 5: [0, 33],
           6: [None, _odd(b["points"])], 8: [S + 1]}
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_lattice_refined(*args))
    f64 = lambda t: _p(t)
    work = b["theta"]
    good = [ctx.handle, 1, C.byref(_field()), C.byref(_params()), f64(b["theta"]), 1, 0.0, 0.0, -1,
            None, 0, 0, None, None, None, 1e-3, f64(work), f64(work), f64(work), f64(work), f64(work),
            None, None, None, None, None]
    bad = {0: [None], 3: [C.byref(_params(lam=0.0))], 4: [None, _odd(b["theta"])], 5: [0], 6: [float("inf")],
           8: [200], 10: [-1], 15: [0.0, -1.0], 16: [None], 17: [None], 18: [None], 19: [None], 20: [None]}
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_jacobian(*args))
    good = [ctx.handle, f64(b["theta"]), 1, f64(work), f64(work), 0.0, None]
    bad = {0: [None], 1: [None, _odd(b["theta"])], 2: [0], 3: [None], 4: [None], 5: [-1.0, float("nan")]}
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_gn_step(*args))
    t = f64(b["theta"])
    good = [ctx.handle, 1, t, t, t, t, t, t, t, t, t, 3.0, 0.5, 0, None]
    bad = {0: [None], 1: [0, (1 << 24) + 1], 2: [None, _odd(b["theta"])], 3: [None], 4: [None], 5: [None],
           6: [None], 7: [None], 8: [None], 9: [None], 10: [None], 11: [0.5, float("inf")],
           12: [0.0, 1.5, float("nan")]}
    for i, vals in bad.items():
        for v in vals:
            args = list(good)
            args[i] = v
            _expect_invalid(L.comet_scan_lm_step(*args))
    _untouched(b)


def test_context_validation():
    L = B.lib()
    h = C.c_void_p()
    _expect_invalid(L.comet_ctx_create(-1, C.byref(h)))
    _expect_invalid(L.comet_ctx_create(torch.cuda.device_count(), C.byref(h)))
    _expect_invalid(L.comet_ctx_create(0, None))
    _expect_invalid(L.comet_ctx_status(None, C.byref(C.c_int32())))
    _expect_invalid(L.comet_ctx_set_copy_wait(None, 0))
    c = B.Context(0)
    _expect_invalid(L.comet_ctx_set_copy_wait(c.handle, -1))
    _expect_invalid(L.comet_ctx_set_dca_ctas_per_sm(None, 1))
    _expect_invalid(L.comet_ctx_set_dca_ctas_per_sm(c.handle, -1))
    _expect_invalid(L.comet_ctx_set_dca_ctas_per_sm(c.handle, 65))
    _expect_invalid(L.comet_ctx_set_dca_chunk_wires(None, 8))
    for w in (-1, 1, 3, 1025):
        _expect_invalid(L.comet_ctx_set_dca_chunk_wires(c.handle, w))
    _expect_invalid(L.comet_ctx_set_record_blocks(None, 1))
    for v in (-1, 2):
        _expect_invalid(L.comet_ctx_set_record_blocks(c.handle, v))
    _expect_invalid(L.comet_ctx_status(c.handle, None))
    _expect_invalid(L.comet_kernel_arch(None))
    c.close()


def test_binding_rejects_mixed_dtypes_and_host_tensors(ctx, bufs):
    """The binding refuses a dtype mismatch between arrays that share the element type T, and host
    tensors, before calling into the library."""
    b = bufs
    f = B.DeviceField()
    p = B.ScanParams(n_steps=8, lam=0.01, tol=1e-6)
    with pytest.raises(TypeError):
        B.comet_scan_propagate(ctx, f, p, b["seeds"], b["charge"], b["points"].double(), b["n_valid"])
    with pytest.raises(TypeError):
        B.comet_scan_dca(ctx, f, p, b["points"], b["n_valid"], b["charge"], b["wires"], b["offs"],
                         b["drift"].double(), b["mask"], b["rss"], b["n_in"], n_wires=W)
    with pytest.raises(ValueError):
        B.comet_scan_select(ctx, b["rss"].cpu(), 1, b["idx"])
    with pytest.raises(TypeError):
        B.comet_scan_select(ctx, b["rss"], 1, b["idx"].int())
    _untouched(b)
