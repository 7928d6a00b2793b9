"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI on inputs that the
generator or the oracle made, and bring results back in the oracle's layouts."""
import numpy as np
import torch

import oracle as O
from paper_1911_09340_gb300 import binding as B


def seen(x, dtype):
    """The values the device path receives for an input given in float64: rounded to float32 for the
    FP32 path (and exactly representable in float64 again), unchanged for FP64.  Parity tests give
    the oracle these same values, so that the comparison measures the arithmetic, not the input
    rounding."""
    x = np.asarray(x, np.float64)
    return x.astype(np.float32).astype(np.float64) if dtype == torch.float32 else x


# Bars of the FP32 path (FP64: 1e-9 m throughout).  DCA: the FP32 track points stay within 1 um of
# FP64 over three turns (tested) and the distance arithmetic adds rounding of a few ulp of metres,
# so 2 um per (seed, wire); the RSS bound follows from it term by term (rss_bound).  Classification:
# bit-identical except hits whose residual |D - r| lies within 1 um of the cutoff.
FP32_DCA_TOL = 2e-6
CLASS_EDGE = {torch.float32: 1e-6, torch.float64: 1e-9}


def both_params(**kw):
    return O.Params(**kw), B.ScanParams(**kw)


def dev_seeds(seeds_aos, dtype):
    return torch.as_tensor(np.ascontiguousarray(np.asarray(seeds_aos).T), dtype=dtype, device="cuda").contiguous()


def dev_wires(wires_soa, dtype, misalign=0, pad_to=4):
    """[6][ldw] device tensor; ``misalign`` shifts the base pointer by that many elements."""
    W = wires_soa.shape[1]
    ldw = max(pad_to, (W + pad_to - 1) // pad_to * pad_to)
    flat = torch.zeros(6 * ldw + misalign, dtype=dtype, device="cuda")
    w = flat[misalign:].view(6, ldw)
    w[:, :W] = torch.as_tensor(np.asarray(wires_soa), dtype=dtype)
    return w


def gpu_propagate(ctx, field, bp, seeds_aos, q, dtype, bounds=None):
    S = seeds_aos.shape[0]
    seeds = dev_seeds(seeds_aos, dtype)
    charge = torch.full((S,), int(q), dtype=torch.int8, device="cuda")
    pts = torch.full((6, bp.n_rec, S), float("nan"), dtype=dtype, device="cuda")
    nv = torch.zeros(S, dtype=torch.int32, device="cuda")
    B.comet_scan_propagate(ctx, field, bp, seeds, charge, pts, nv, bounds=bounds)
    return seeds, charge, pts, nv


def to_aos_points(pts):
    return pts.double().cpu().numpy().transpose(2, 1, 0)


def gpu_dca(ctx, field, bp, seeds_aos, q, wires_soa, offs, drift, mask, dtype, want_dca=True,
            misalign=0, use_bounds=True):
    bounds = (torch.full(B.bounds_shape(seeds_aos.shape[0]), float("nan"), dtype=torch.float32,
                         device="cuda") if use_bounds else None)
    seeds, charge, pts, nv = gpu_propagate(ctx, field, bp, seeds_aos, q, dtype, bounds=bounds)
    S = seeds_aos.shape[0]
    W = wires_soa.shape[1]
    w = dev_wires(wires_soa, dtype, misalign)
    o = torch.as_tensor(np.asarray(offs, np.int32), device="cuda")
    d = torch.as_tensor(np.asarray(drift), dtype=dtype, device="cuda")
    m = torch.as_tensor(np.asarray(mask, np.uint8), device="cuda")
    rss = torch.full((S,), float("nan"), dtype=dtype, device="cuda")
    n_in = torch.full((S,), -1, dtype=torch.int32, device="cuda")
    dca = torch.full((max(W, 1), S), float("nan"), dtype=dtype, device="cuda") if want_dca else None
    nunc = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.comet_scan_dca(ctx, field, bp, pts, nv, charge, w, o, d, m, rss, n_in, dca_out=dca,
                     n_unconverged=nunc, n_wires=W, bounds=bounds)
    torch.cuda.synchronize()
    out = dict(rss=rss.double().cpu().numpy(), n_in=n_in.cpu().numpy(), n_unconv=int(nunc.item()),
               pts=pts, nv=nv, charge=charge, w=w, o=o, d=d, m=m, bounds=bounds)
    if want_dca:
        out["dca"] = dca[:W].double().cpu().numpy().T   # [S][W]
    return out


def per_wire_residual(dca_sw, offs, drift, mask):
    """min over unmasked hits of |D - r| per (seed, wire); inf where a wire has no unmasked hit."""
    S, W = dca_sw.shape
    e = np.full((S, W), np.inf)
    for i in range(W):
        for j in range(offs[i], offs[i + 1]):
            if not mask[j]:
                e[:, i] = np.minimum(e[:, i], np.abs(dca_sw[:, i] - drift[j]))
    return e


def rss_bound(e_oracle, lam, delta, fp32=True):
    """Largest |RSS_gpu - RSS_oracle| when every DCA is within delta: wires capped with margin
    contribute nothing, the others at most 2*min(e, lam)*delta + delta^2 each; in FP32 add the
    rounding of each squared term (half an ulp of lambda^2 at most) and of the FP32 result."""
    near = e_oracle < lam + delta
    b = np.where(near, 2.0 * np.minimum(e_oracle, lam) * delta + delta * delta, 0.0).sum(1)
    if fp32:
        terms = np.isfinite(e_oracle).sum(1)
        rss = (np.minimum(np.where(np.isfinite(e_oracle), e_oracle, 0.0), lam) ** 2).sum(1)
        b = b + terms * 6e-8 * lam * lam + 1.2e-7 * rss
    return b
