"""Smoothed RSS, residual Jacobians and Gauss-Newton steps (comet_scan_jacobian, comet_scan_gn_step).

CPU: the oracle's smoothed RSS tends to Eq. 1's capped RSS as tau -> 0.  GPU (FP64): the DCAs equal
the oracle's; dD/dtheta equals central finite differences of the oracle's DCAs (rel 1e-4); the
smoothed RSS equals the oracle's and its gradient the finite differences of the oracle's; Gauss-
Newton from a seed half a lattice step off lowers the smoothed RSS and the momentum error.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1911_09340_gb300 import synth

UNIFORM = synth.uniform_field(1.0)


def _truth_theta(ev):
    return np.array([ev.vertex[2], ev.phi0, ev.pz, ev.pt])


def test_smoothed_rss_tends_to_the_capped_rss():
    ev = synth.single_event_fp64()
    th = np.stack([_truth_theta(ev), _truth_theta(ev) + [0.004, 0.003, 0.4, 0.6]])
    mask = np.zeros(ev.n_hits, np.uint8)
    for lam in (8e-4, 1e-2):
        P = O.Params(n_steps=ev.n_steps[0], stride=16, lam=lam, tol=1e-12)
        s0, D = O.smoothed_rss(UNIFORM, P, th, ev.vertex[0], ev.vertex[1], -1, O.wires_aos(ev.wires),
                               ev.hit_offsets, ev.drift, mask, 1e-12)
        r = O.scan(UNIFORM, P, O.seeds_from_theta(th, ev.vertex[0], ev.vertex[1]), -1,
                   O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, mask)
        assert np.allclose(s0, r["rss"], rtol=1e-12, atol=0)
        # each smoothed term is a convex combination of e^2 and lam^2, so never below the capped
        # term min(e^2, lam^2): a wide smoothing can only raise the sum
        s1, _ = O.smoothed_rss(UNIFORM, P, th, ev.vertex[0], ev.vertex[1], -1, O.wires_aos(ev.wires),
                               ev.hit_offsets, ev.drift, mask, 1e-3)
        assert np.all(s1 >= s0 * (1 - 1e-12))


# ------------------------------------------------------------------------------------------------
# GPU
# ------------------------------------------------------------------------------------------------

def _gpu_eval(ctx, ev, theta, stride, lam, tau, want=True):
    import torch
    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import scan
    f64 = dict(dtype=torch.float64, device="cuda")
    S = theta.shape[0]
    dev = scan.DeviceEvent.from_event(ev, torch.float64)
    p = B.ScanParams(n_steps=ev.n_steps[0], stride=stride, lam=lam, tol=1e-12)
    th = torch.as_tensor(theta, **f64).contiguous()
    W = dev.W
    work = torch.empty(S * W * B.JAC_WORK_PER_PAIR, **f64)
    srss, grad = torch.empty(S, **f64), torch.empty((S, 4), **f64)
    jtj, jtr = torch.empty((S, 16), **f64), torch.empty((S, 4), **f64)
    D, J = torch.empty((S, W), **f64), torch.empty((S, W, 4), **f64)
    B.comet_scan_jacobian(ctx, B.DeviceField.from_synth(UNIFORM), p, th, ev.vertex[0], ev.vertex[1], -1,
                          dev.wires, dev.hit_offsets, dev.drift, dev.mask, tau, work, srss, grad, jtj,
                          jtr, dca_out=D, jac_out=J, n_wires=W)
    torch.cuda.synchronize()
    return (srss.cpu().numpy(), grad.cpu().numpy(), D.cpu().numpy(), J.cpu().numpy(),
            jtj.cpu().numpy(), jtr.cpu().numpy())


@pytest.mark.gpu
@pytest.mark.parametrize("stride", [1, 16])
def test_dca_and_jacobian_match_oracle_and_finite_differences(ctx, stride):
    ev = synth.single_event_fp64()
    t0 = _truth_theta(ev)
    theta = np.stack([t0, t0 + [0.002, -0.002, 0.3, -0.4], t0 + [-0.003, 0.001, -0.2, 0.5]])
    lam, tau = 8e-4, 1e-3
    srss, grad, D, J, _, _ = _gpu_eval(ctx, ev, theta, stride, lam, tau)
    P = O.Params(n_steps=ev.n_steps[0], stride=stride, lam=lam, tol=1e-12)
    mask = np.zeros(ev.n_hits, np.uint8)
    args = (ev.vertex[0], ev.vertex[1], -1, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, mask)
    o_srss, o_D = O.smoothed_rss(UNIFORM, P, theta, *args, tau)
    near = o_D < 0.02
    assert np.abs(D[near] - o_D[near]).max() <= 1e-9
    assert np.allclose(srss, o_srss, rtol=1e-8, atol=1e-14)
    eps = np.array([1e-6, 1e-6, 1e-4, 1e-4])
    for k in range(4):
        tp, tm = theta.copy(), theta.copy()
        tp[:, k] += eps[k]
        tm[:, k] -= eps[k]
        sp, Dp = O.smoothed_rss(UNIFORM, P, tp, *args, tau)
        sm, Dm = O.smoothed_rss(UNIFORM, P, tm, *args, tau)
        Jfd = (Dp - Dm) / (2 * eps[k])
        scale = np.abs(Jfd[near]).max()
        assert np.abs(J[..., k][near] - Jfd[near]).max() <= 1e-4 * scale, k
        gfd = (sp - sm) / (2 * eps[k])
        assert np.allclose(grad[:, k], gfd, rtol=1e-4, atol=1e-4 * np.abs(gfd).max() + 1e-15), k


@pytest.mark.gpu
def test_gauss_newton_improves_a_seed_half_a_step_off(ctx):
    import torch
    from paper_1911_09340_gb300 import experiments as X
    ev = synth.single_event_fp64()
    spec = ev.partitions[0]
    step = np.array([2 * h / (n - 1) for h, n in zip(spec.half_width, spec.counts)])
    t0 = _truth_theta(ev)
    # half a lattice step off in every parameter (inside the basin; a full step off at a sub-mm
    # cutoff leaves almost every residual beyond the cap and Gauss-Newton may settle elsewhere)
    start = np.stack([t0 + 0.5 * step * [1, -1, 1, 1], t0 + 0.5 * step * [-1, 1, 0, -1]])
    G = X.GaussNewton(ctx, ev, 0, stride=16, lam=1e-2, tau=1e-3, K=2)
    G.theta.copy_(torch.as_tensor(start))
    G.evaluate()
    s_start = G.srss.cpu().numpy().copy()
    G.run(iters=10)
    s_end = G.srss.cpu().numpy()
    th = G.theta.cpu().numpy()
    assert np.all(s_end <= s_start)
    p_true = math.hypot(ev.pt, ev.pz)
    dp_start = np.abs(np.hypot(start[:, 2], start[:, 3]) - p_true)
    dp_end = np.abs(np.hypot(th[:, 2], th[:, 3]) - p_true)
    assert np.all(dp_end < dp_start)


@pytest.mark.gpu
def test_lm_step_accepts_lower_trials_and_solves_the_damped_system(ctx):
    """comet_scan_lm_step on hand-made normal equations: a trial of lower smoothed RSS replaces the
    current seed (theta, srss, JTJ, JTR) and shrinks mu, a higher one is rejected and grows mu; the
    next trial solves (JTJ + mu diag JTJ) delta = -JTR (numpy), and a seed whose matrix is not
    positive definite gets delta = 0."""
    import torch
    from paper_1911_09340_gb300 import binding as B
    rng = np.random.default_rng(4)
    S = 3
    f64 = dict(dtype=torch.float64, device="cuda")
    M = rng.normal(size=(S, 4, 4))
    jtj = np.einsum("sij,skj->sik", M, M) + 0.1 * np.eye(4)
    jtj_t = np.einsum("sij,skj->sik", M[::-1], M[::-1]) + 0.2 * np.eye(4)
    jtj_t[2] = -np.eye(4)                                   # seed 2's trial: not positive definite
    theta, theta_t = rng.normal(size=(S, 4)), rng.normal(size=(S, 4))
    jtr, jtr_t = rng.normal(size=(S, 4)), rng.normal(size=(S, 4))
    srss = np.array([1.0, 1.0, 1.0])
    srss_t = np.array([0.5, 2.0, 0.25])                     # accept, reject, accept
    mu = np.array([1e-3, 1e-3, 1e-3])
    d = {k: torch.as_tensor(np.ascontiguousarray(v), **f64) for k, v in dict(
        theta=theta, srss=srss, jtj=jtj.reshape(S, 16), jtr=jtr, theta_t=theta_t, srss_t=srss_t,
        jtj_t=jtj_t.reshape(S, 16), jtr_t=jtr_t, mu=mu).items()}
    B.comet_scan_lm_step(ctx, d["theta"], d["srss"], d["jtj"], d["jtr"], d["theta_t"], d["srss_t"],
                         d["jtj_t"], d["jtr_t"], d["mu"], up=4.0, down=0.25)
    acc = srss_t < srss
    cur_theta = np.where(acc[:, None], theta_t, theta)
    cur_jtj = np.where(acc[:, None, None], jtj_t, jtj)
    cur_jtr = np.where(acc[:, None], jtr_t, jtr)
    new_mu = np.where(acc, mu * 0.25, mu * 4.0)
    assert np.array_equal(d["srss"].cpu().numpy(), np.minimum(srss, srss_t))
    assert np.array_equal(d["theta"].cpu().numpy(), cur_theta)
    assert np.allclose(d["mu"].cpu().numpy(), new_mu, rtol=1e-15)
    nxt = d["theta_t"].cpu().numpy()
    for s in range(S):
        A = cur_jtj[s] + new_mu[s] * np.diag(np.diag(cur_jtj[s]))
        if np.all(np.linalg.eigvalsh(A) > 0):
            want = cur_theta[s] + np.linalg.solve(A, -cur_jtr[s])
        else:
            want = cur_theta[s]
        assert np.allclose(nxt[s], want, rtol=1e-10, atol=1e-12), s
    with pytest.raises(B.CometError):
        B.comet_scan_lm_step(ctx, d["theta"], d["srss"], d["jtj"], d["jtr"], d["theta_t"], None, None,
                             None, d["mu"], up=0.5)


@pytest.mark.gpu
def test_levenberg_marquardt_never_raises_the_smoothed_rss(ctx):
    """Levenberg-Marquardt from seeds half and a whole lattice step off: the smoothed RSS of the kept
    seeds never increases from iteration to iteration, ends below its start, and the momentum error
    of a seed half a step off shrinks."""
    import torch
    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import experiments as X
    ev = synth.single_event_fp64()
    spec = ev.partitions[0]
    step = np.array([2 * h / (n - 1) for h, n in zip(spec.half_width, spec.counts)])
    t0 = _truth_theta(ev)
    start = np.stack([t0 + 0.5 * step * [1, -1, 1, 1], t0 + step * [-1, 1, 1, -1]])
    G = X.GaussNewton(ctx, ev, 0, stride=16, lam=8e-4, tau=1e-3, K=2)
    G.theta.copy_(torch.as_tensor(start))
    G.run_lm(iters=0)
    hist = [G.srss.cpu().numpy().copy()]
    for _ in range(8):
        G._eval_at(G.t_theta, G.t_srss, G.t_grad, G.t_jtj, G.t_jtr)
        B.comet_scan_lm_step(ctx, G.theta, G.srss, G.jtj, G.jtr, G.t_theta, G.t_srss, G.t_jtj, G.t_jtr,
                             G.mu)
        hist.append(G.srss.cpu().numpy().copy())
    hist = np.array(hist)
    assert np.all(np.diff(hist, axis=0) <= 0)
    assert np.all(hist[-1] < hist[0])
    th = G.theta.cpu().numpy()
    p_true = math.hypot(ev.pt, ev.pz)
    assert abs(math.hypot(th[0, 2], th[0, 3]) - p_true) < abs(math.hypot(start[0, 2], start[0, 3]) - p_true)


@pytest.mark.gpu
def test_gradient_in_the_six_cartesian_seed_components(ctx):
    """d(smoothed RSS)/d(x, y, z, px, py, pz) of the seed against central finite differences of the
    oracle's smoothed RSS of Cartesian seeds (rel 1e-4)."""
    import torch
    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import scan
    ev = synth.single_event_fp64()
    t0 = _truth_theta(ev)
    theta = np.stack([t0, t0 + [0.002, -0.002, 0.3, -0.4]])
    lam, tau, stride = 8e-4, 1e-3, 16
    f64 = dict(dtype=torch.float64, device="cuda")
    dev = scan.DeviceEvent.from_event(ev, torch.float64)
    p = B.ScanParams(n_steps=ev.n_steps[0], stride=stride, lam=lam, tol=1e-12)
    S, W = theta.shape[0], dev.W
    th = torch.as_tensor(theta, **f64).contiguous()
    outs = [torch.empty(S * W * B.JAC_WORK_PER_PAIR, **f64), torch.empty(S, **f64), torch.empty((S, 4), **f64),
            torch.empty((S, 16), **f64), torch.empty((S, 4), **f64)]
    g6 = torch.empty((S, 6), **f64)
    B.comet_scan_jacobian(ctx, B.DeviceField.from_synth(UNIFORM), p, th, ev.vertex[0], ev.vertex[1], -1,
                          dev.wires, dev.hit_offsets, dev.drift, dev.mask, tau, *outs, n_wires=W, grad6=g6)
    g6 = g6.cpu().numpy()
    P = O.Params(n_steps=ev.n_steps[0], stride=stride, lam=lam, tol=1e-12)
    args = (-1, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, np.zeros(ev.n_hits, np.uint8), tau)
    seeds = O.seeds_from_theta(theta, ev.vertex[0], ev.vertex[1])
    eps = [1e-6, 1e-6, 1e-6, 1e-4, 1e-4, 1e-4]
    for k in range(6):
        sp, sm = seeds.copy(), seeds.copy()
        sp[:, k] += eps[k]
        sm[:, k] -= eps[k]
        fd = (O.smoothed_rss_seeds(UNIFORM, P, sp, *args)[0] - O.smoothed_rss_seeds(UNIFORM, P, sm, *args)[0]) / (2 * eps[k])
        assert np.allclose(g6[:, k], fd, rtol=1e-4, atol=1e-4 * np.abs(fd).max() + 1e-15), (k, g6[:, k], fd)


@pytest.mark.gpu
def test_smoothed_rss_autograd_functions(ctx):
    """torch.autograd through the smoothed RSS: backward of SmoothedRSS gives the kernel's gradient
    in theta (scaled by the incoming gradient), SmoothedRSSCartesian the six-component one, and the
    latter equals central finite differences of the oracle's smoothed RSS of Cartesian seeds."""
    import torch
    from paper_1911_09340_gb300 import autodiff as A
    from paper_1911_09340_gb300 import binding as B
    from paper_1911_09340_gb300 import scan
    ev = synth.single_event_fp64()
    t0 = _truth_theta(ev)
    theta_np = np.stack([t0, t0 + [0.002, -0.002, 0.3, -0.4], t0 + [-0.001, 0.001, -0.2, 0.2]])
    lam, tau, stride = 8e-4, 1e-3, 16
    spec = A.SmoothedRSSSpec(ctx, B.DeviceField.from_synth(UNIFORM),
                             B.ScanParams(n_steps=ev.n_steps[0], stride=stride, lam=lam, tol=1e-12),
                             scan.DeviceEvent.from_event(ev, torch.float64), -1, tau)
    theta = torch.tensor(theta_np, dtype=torch.float64, device="cuda", requires_grad=True)
    s = A.SmoothedRSS.apply(theta, spec, ev.vertex[0], ev.vertex[1])
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    (s * w).sum().backward()
    srss, grad, grad6 = A._evaluate(spec, theta.detach(), ev.vertex[0], ev.vertex[1])
    assert torch.equal(s.detach(), srss)
    assert torch.equal(theta.grad, w[:, None] * grad)

    seeds_np = O.seeds_from_theta(theta_np, ev.vertex[0], ev.vertex[1])
    seeds = torch.tensor(seeds_np, dtype=torch.float64, device="cuda", requires_grad=True)
    s6 = A.SmoothedRSSCartesian.apply(seeds, spec)
    s6.sum().backward()
    assert torch.allclose(s6.detach(), srss, rtol=1e-12, atol=0)
    g6 = seeds.grad.cpu().numpy()
    P = O.Params(n_steps=ev.n_steps[0], stride=stride, lam=lam, tol=1e-12)
    args = (-1, O.wires_aos(ev.wires), ev.hit_offsets, ev.drift, np.zeros(ev.n_hits, np.uint8), tau)
    eps = [1e-6, 1e-6, 1e-6, 1e-4, 1e-4, 1e-4]
    for k in range(6):
        sp, sm = seeds_np.copy(), seeds_np.copy()
        sp[:, k] += eps[k]
        sm[:, k] -= eps[k]
        fd = (O.smoothed_rss_seeds(UNIFORM, P, sp, *args)[0] - O.smoothed_rss_seeds(UNIFORM, P, sm, *args)[0]) / (2 * eps[k])
        assert np.allclose(g6[:, k], fd, rtol=1e-4, atol=1e-4 * np.abs(fd).max() + 1e-15), (k, g6[:, k], fd)
    with pytest.raises(ValueError):
        A.SmoothedRSSCartesian.apply(seeds.detach() + torch.tensor([0.0, 1e-3, 0, 0, 0, 0], device="cuda",
                                                                    dtype=torch.float64) * torch.arange(3, device="cuda", dtype=torch.float64)[:, None], spec)
