"""GPU parity at full workload sizes (sampled outputs against the oracle's direct sums), the adjoint,
autograd and Gaussian smoothing."""
import math

import numpy as np
import pytest

import paper_2110_11866_gb300 as m
import workloads as WL
from oracle import morlet as om
from oracle import sft_dd
from tests.gpu_helpers import gpu_forward, oracle_forward, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _sample_idx(N, L, rng, n=24):
    """Sampled output indices: both ends (boundary windows), tile edges and random interior points."""
    fixed = [0, 1, N - 1, N - 2, min(N - 1, L), min(N - 1, 4095), min(N - 1, 4096), N // 2]
    return np.unique(np.concatenate([fixed, rng.integers(0, N, n)]))


def _row_errors(got, ref):
    """Per-row error max|got - ref| / max|ref| of [rows, n] arrays (the oracle's max in the denominator)."""
    return np.abs(got - ref).max(axis=1) / np.maximum(np.abs(ref).max(axis=1), 1e-300)


def test_c3_scalogram_full_size_every_element():
    """Config 3 at full size (256 ragged signals x 32 scales, 1.27 G outputs), compensated FP32, in the
    bench's launch configuration (autotuned schedule, one graph-captured forward). Every output of
    every (signal, scale) row is compared with the oracle's O-SFT (the double-double kernel integral
    of Sec. II-B with the oracle's own fit), in groups of signals; a row's error is
    max|W_gpu - W_oracle| / max|W_oracle| over the row, gate 1e-5."""
    import torch
    w = WL.c3_scalogram()
    sigmas, lens = w.sigmas, w.lengths
    S = len(sigmas)
    fits = [om.fit_direct(s, 6.0, 4) for s in sigmas]
    x = torch.from_numpy(w.concat()).cuda()
    plan = m.morlet_plan(lens, sigmas, K=4, precision=m.MORLET_FP32_COMP, flags=m.MORLET_FLAG_AUTOTUNE)
    W = torch.empty(sum(lens) * S, dtype=torch.complex64, device="cuda")
    m.morlet_forward(plan, x, W)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    offs = np.concatenate([[0], np.cumsum(lens)])
    worst, where, rows = 0.0, None, 0
    g0 = 0
    while g0 < len(lens):
        g1 = g0 + 1
        while g1 < len(lens) and offs[g1 + 1] - offs[g0] <= (4 << 20):
            g1 += 1
        ref, _ = sft_dd.sft_batch(w.signals[g0:g1], fits)
        got = W[S * int(offs[g0]):S * int(offs[g1])].cpu().numpy()
        o = 0
        for i in range(g0, g1):
            n = lens[i]
            e = _row_errors(got[o:o + S * n].reshape(S, n), ref[o:o + S * n].reshape(S, n))
            rows += S
            if e.max() > worst:
                worst, where = float(e.max()), (i, int(np.argmax(e)))
            o += S * n
        del ref, got
        g0 = g1
    print(f"c3 full size, every element: worst row error {worst:.3e} (signal, scale) = {where}, {rows} rows, "
          f"schedule {m.morlet_plan_schedule(plan)}")
    assert rows == len(lens) * S
    assert worst < 1e-5
    del W


@pytest.fixture(scope="module")
def c5_oracle():
    """The oracle's O-SFT of the whole config-5 signal at its three scales (K = 6), three chains in
    parallel."""
    x = WL.c5_pink()
    fits = [om.fit_direct(s, 6.0, 6) for s in WL.C5_SIGMAS]
    W, _ = sft_dd.sft_batch([x.astype(np.float64)], fits)
    return x, fits, W.reshape(len(fits), len(x))


@pytest.mark.parametrize("s", range(len(WL.C5_SIGMAS)))
def test_c5_long_signal_every_element(c5_oracle, s):
    """Config 5: one 2^24-sample pink-noise signal, K = 6, compensated FP32 (gate 1e-5) and FP64 (gate
    1e-12): every output against the oracle's O-SFT (multi-tile carries and prefix sums at large n),
    error over max|W_oracle|; a few outputs also against the direct sum of the fitted kernel."""
    x, fits, refs = c5_oracle
    sigma, ref = WL.C5_SIGMAS[s], refs[s]
    N = len(x)
    idx = np.array([0, N // 3, N - 17, N - 1, 12345678])
    direct = om.morlet_sft_direct(x.astype(np.float64), fits[s], idx)
    assert np.abs(direct - ref[idx]).max() <= 1e-12 * np.abs(ref).max()
    for prec, tol in ((m.MORLET_FP32_COMP, 1e-5), (m.MORLET_FP64, 1e-12)):
        xs = x.astype(np.float64) if prec == m.MORLET_FP64 else x
        plan, out = gpu_forward([xs], [sigma], K=6, precision=prec)
        e = float(np.abs(out[0][0] - ref).max() / np.abs(ref).max())
        print(f"c5 sigma={sigma} precision={prec}: every element, rel err {e:.3e}")
        assert e < tol
        del out


def _loss_terms(W, wts):
    return wts * np.log(1e-6 + np.abs(W) ** 2)


def test_c4_adjoint_vs_direct_and_finite_differences():
    """Config 4: batch 64 x 65536, 16 scales, K = 4; loss = sum w log(1e-6 + |W|^2).
    (a) FP32-compensated adjoint against the oracle's adjoint, every coordinate of 8 signals (the sum
        over the 16 scales of the kernel-integral adjoint, itself pinned against the direct
        transpose), tolerance 1e-5 of the oracle's max |gx| per signal; sampled coordinates also
        against the direct transpose;
    (b) FP64 adjoint against central finite differences (eps = 1e-6) of the FP64 transform on 32
        random coordinates; each loss difference is summed over the outputs the coordinate touches
        (|n - t| <= L_s per scale), so that rounding of the 67 M-term sum does not swamp it."""
    import torch
    w = WL.c4_batch()
    wts = WL.c4_loss_weights()
    sig = w.sigmas
    S, B, N = len(sig), len(w.signals), len(w.signals[0])
    fits = [om.fit_direct(s, 6.0, 4) for s in sig]
    xb = np.stack(w.signals)
    wt = torch.from_numpy(wts).cuda()

    def grad_W(W):  # dLoss/dRe W + i dLoss/dIm W, laid out [signal][scale][n]
        Wv = W.view(B, S, N)
        return (wt * 2 * Wv / (1e-6 + Wv.abs() ** 2)).reshape(-1)

    # (a) compensated FP32
    plan = m.morlet_plan([N] * B, sig, K=4, precision=m.MORLET_FP32_COMP)
    x = torch.from_numpy(xb.reshape(-1)).cuda()
    W = torch.empty(B * S * N, dtype=torch.complex64, device="cuda")
    m.morlet_forward(plan, x, W)
    g = grad_W(W).to(torch.complex64).contiguous()
    gx = torch.empty(B * N, dtype=torch.float32, device="cuda")
    m.morlet_backward(plan, g, gx)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    rng = np.random.default_rng(7)
    gh = g.view(B, S, N).cpu().numpy().astype(np.complex128)
    gxh = gx.view(B, N).cpu().numpy()
    worst, worst_direct = 0.0, 0.0
    for b in rng.choice(B, 8, replace=False):
        ref = sum(sft_dd.adjoint_sft(gh[b, s], fits[s]) for s in range(S))
        worst = max(worst, float(np.abs(gxh[b] - ref).max() / np.abs(ref).max()))
        idx = _sample_idx(N, fits[-1]["L"], rng, n=6)
        refd = sum(om.adjoint_direct(gh[b, s], fits[s], idx) for s in range(S))
        worst_direct = max(worst_direct, float(np.abs(gxh[b, idx] - refd).max() / np.abs(ref).max()))
    print(f"c4 adjoint fp32-comp vs oracle adjoint: every coordinate {worst:.3e}, sampled direct {worst_direct:.3e}")
    assert worst < 1e-5 and worst_direct < 1e-5

    # (b) FP64 adjoint vs central differences of the FP64 forward
    plan64 = m.morlet_plan([N] * B, sig, K=4, precision=m.MORLET_FP64)
    x64 = torch.from_numpy(xb.reshape(-1).astype(np.float64)).cuda()
    W64 = torch.empty(B * S * N, dtype=torch.complex128, device="cuda")
    m.morlet_forward(plan64, x64, W64)
    g64 = grad_W(W64).to(torch.complex128).contiguous()
    gx64 = torch.empty(B * N, dtype=torch.float64, device="cuda")
    m.morlet_backward(plan64, g64, gx64)
    torch.cuda.synchronize()
    Ls = [f["L"] for f in fits]
    eps = 1e-6
    Wp = torch.empty_like(W64)
    Wm = torch.empty_like(W64)
    worst_fd = 0.0
    for _ in range(32):
        b, t = int(rng.integers(B)), int(rng.integers(N))
        xp = x64.clone()
        xp[b * N + t] += eps
        xm = x64.clone()
        xm[b * N + t] -= eps
        m.morlet_forward(plan64, xp, Wp)
        m.morlet_forward(plan64, xm, Wm)
        d = 0.0
        for s in range(S):
            lo, hi = max(0, t - Ls[s]), min(N, t + Ls[s] + 1)
            base = (b * S + s) * N
            lp = torch.log(1e-6 + Wp[base + lo:base + hi].abs() ** 2)
            lm = torch.log(1e-6 + Wm[base + lo:base + hi].abs() ** 2)
            d += float((wt[b, s, lo:hi].double() * (lp - lm)).sum().item())
        fd = d / (2 * eps)
        an = float(gx64[b * N + t].item())
        worst_fd = max(worst_fd, abs(fd - an) / (abs(an) + 1e-3 * float(gx64.abs().max().item())))
    print(f"c4 adjoint fp64 vs central differences: worst rel {worst_fd:.3e}")
    assert worst_fd < 1e-5


@pytest.mark.parametrize("precision,form", [(m.MORLET_FP32_COMP, m.MORLET_FORM_ROTATING),
                                            (m.MORLET_FP32_COMP, m.MORLET_FORM_KERNEL),
                                            (m.MORLET_FP32_PLAIN, m.MORLET_FORM_ROTATING),
                                            (m.MORLET_FP64, m.MORLET_FORM_ROTATING)])
def test_backward_every_coordinate(precision, form):
    """morlet_backward on a ragged batch (rows shorter than the window, rows of window segments and of
    start-state items, every alignment) in each precision and form, against the oracle's adjoint
    (sum over scales of the kernel-integral adjoint) at every coordinate; gate 1e-5 of max|gx|
    (1e-12 in FP64, 1e-3 in plain FP32). Two calls with the same buffers replay one graph."""
    import torch
    rng = np.random.default_rng(31 + precision + 3 * form)
    lens = [1, 70001, 4097, 300000, 999]
    sigmas = [8.0, 100.0, 700.0, 3000.0, 9000.0]
    S, n_in = len(sigmas), sum(lens)
    f64 = precision == m.MORLET_FP64
    plan = m.morlet_plan(lens, sigmas, K=4, precision=precision, form=form)
    g = (rng.standard_normal(n_in * S) + 1j * rng.standard_normal(n_in * S))
    gt = torch.from_numpy(g.astype(np.complex128 if f64 else np.complex64)).cuda()
    gx = torch.full((n_in,), float("nan"), dtype=torch.float64 if f64 else torch.float32, device="cuda")
    for _ in range(2):
        m.morlet_backward(plan, gt, gx)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    gxh = gx.cpu().numpy()
    gh = gt.cpu().numpy().astype(np.complex128)
    fits = [om.fit_direct(sg, 6.0, 4) for sg in sigmas]
    tol = {m.MORLET_FP32_COMP: 1e-5, m.MORLET_FP32_PLAIN: 1e-3, m.MORLET_FP64: 1e-12}[precision]
    off = 0
    for n in lens:
        ref = sum(sft_dd.adjoint_sft(gh[S * off + s * n: S * off + (s + 1) * n], fits[s]) for s in range(S))
        e = rel_err(gxh[off:off + n], ref)
        assert e < tol, (n, e)
        off += n
    with pytest.raises(m.MorletError) as err:
        p2 = m.morlet_plan(lens, sigmas, K=4, precision=precision, flags=m.MORLET_FLAG_NO_ADJOINT)
        m.morlet_backward(p2, gt, gx)
    assert err.value.code == m.MORLET_ERR_UNSUPPORTED


def test_autograd_function_matches_backward():
    import torch
    from paper_2110_11866_gb300.torch_ops import MorletFn, MorletTransform
    rng = np.random.default_rng(3)
    lens = [5000, 12000]
    tr = MorletTransform(lens, [10.0, 80.0], K=4, precision=m.MORLET_FP32_COMP)
    x = torch.from_numpy(rng.standard_normal(sum(lens)).astype(np.float32)).cuda().requires_grad_(True)
    W = MorletFn.apply(x, tr)
    wts = torch.from_numpy(rng.standard_normal(W.numel()).astype(np.float32)).cuda()
    loss = (wts * torch.log(1e-6 + W.abs() ** 2)).sum()
    loss.backward()
    g = (wts * 2 * W / (1e-6 + W.abs() ** 2)).detach().to(torch.complex64)
    gx = tr.backward(g)
    torch.cuda.synchronize()
    assert torch.allclose(x.grad, gx, rtol=0, atol=1e-6 * float(gx.abs().max()))


@pytest.mark.parametrize("deriv", [0, 1, 2])
@pytest.mark.parametrize("precision", [m.MORLET_FP32_COMP, m.MORLET_FP64])
def test_gauss_smooth(deriv, precision):
    """gauss_smooth (eq. GsSFT and its derivative forms) against the oracle's kernel integral."""
    import torch
    rng = np.random.default_rng(deriv)
    N = 70000
    x = rng.standard_normal(N)
    for sigma, P in ((5.0, 3), (40.0, 4), (700.0, 6)):
        gf = om.fit_gauss(sigma, P, deriv)
        ref = sft_dd.sft_gauss(x, gf)
        dt = torch.float64 if precision == m.MORLET_FP64 else torch.float32
        xt = torch.from_numpy(x).to(dt).cuda()
        y = torch.empty(N, dtype=dt, device="cuda")
        m.gauss_smooth(xt, N, sigma, P, deriv, precision, y)
        torch.cuda.synchronize()
        if precision != m.MORLET_FP64:
            ref = sft_dd.sft_gauss(x.astype(np.float32).astype(np.float64), gf)
        e = rel_err(y.cpu().numpy(), ref)
        print(f"gauss deriv={deriv} sigma={sigma} P={P} precision={precision}: {e:.2e}")
        assert e < (1e-12 if precision == m.MORLET_FP64 else 1e-5)


@pytest.mark.parametrize("deriv", [0, 1, 2])
def test_gauss_smooth_start_state_everywhere(deriv):
    """Gaussian smoothing by the SFT (compensated FP32, a ragged batch at several scales) with every
    row on start-state items (thresholds 0:1, 64-tile items longest first, the schedule the
    autotuner may pick for these plans) against the oracle's kernel integral, gate 1e-5."""
    import torch
    rng = np.random.default_rng(60 + deriv)
    lens = [70000, 5, 4097, 30000]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    sigmas, P = [5.0, 40.0, 700.0], 6
    plan = m.morlet_plan(lens, sigmas, K=P + 1, method=m.MORLET_GAUSS, deriv=deriv, precision=m.MORLET_FP32_COMP)
    m.morlet_plan_set_row_thresholds(plan, 0, 1)
    m.morlet_plan_set_schedule(plan, 16, 64, 2, 0)
    st = m.morlet_plan_stats(plan)
    assert st["rows_start_state"] == len(lens) * len(sigmas), st
    S, n_in = len(sigmas), sum(lens)
    y = torch.full((n_in * S,), float("nan"), dtype=torch.float32, device="cuda")
    m.morlet_forward(plan, torch.from_numpy(np.concatenate(sigs)).cuda(), y)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    yh = y.cpu().numpy()
    off = 0
    for x, n in zip(sigs, lens):
        for s, sg in enumerate(sigmas):
            gf = om.fit_gauss(sg, P, deriv)
            ref = sft_dd.sft_gauss(x.astype(np.float64), gf)
            got = yh[S * off + s * n: S * off + (s + 1) * n]
            scale = np.abs(ref).max()
            if n < 2 * gf["L"]:  # a row shorter than the window: the rounding scale of its arithmetic
                scale = max(scale, np.abs(om.kernel_gauss(gf)).sum() * np.abs(x).max())
            e = float(np.abs(got - ref).max() / scale)
            assert e < 1e-5, (deriv, n, sg, e)
        off += n


@pytest.mark.parametrize("deriv", [0, 1, 2])
def test_gauss_smooth_asft(deriv):
    """Gaussian smoothing and its derivatives by the ASFT (eqs. GsASFT, gddAsft, FP32 attenuated
    recursion): a batch of ragged signals at several scales against the oracle's double-double
    recursion with the oracle's own fit; the ASFT gate 1e-4 of max|y|."""
    import torch
    rng = np.random.default_rng(20 + deriv)
    lens = [70000, 5, 4097, 30000]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    sigmas = [5.0, 24.0, 40.0, 700.0]
    P = 6
    plan = m.morlet_plan(lens, sigmas, K=P + 1, method=m.MORLET_GAUSS, transform=m.MORLET_ASFT,
                         deriv=deriv, precision=m.MORLET_FP32_PLAIN)
    # the damped window sum forgets everything older than 2L + 1 samples: every row (L <= 2800) runs
    # as restarted window segments, none as a look-back chain
    st = m.morlet_plan_stats(plan)
    assert st["rows_lookback"] == 0 and st["rows_window"] == len(lens) * len(sigmas), st
    S, n_in = len(sigmas), sum(lens)
    xt = torch.from_numpy(np.concatenate(sigs)).cuda()
    y = torch.full((n_in * S,), float("nan"), dtype=torch.float32, device="cuda")
    m.morlet_forward(plan, xt, y)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    yh = y.cpu().numpy()
    off = 0
    for x, n in zip(sigs, lens):
        for s, sigma in enumerate(sigmas):
            gf = om.fit_gauss_asft(sigma, P, deriv, om.default_n0(sigma))
            ref = sft_dd.asft_gauss(x.astype(np.float64), gf)
            got = yh[S * off + s * n: S * off + (s + 1) * n]
            e = rel_err(got, ref)
            print(f"gauss asft deriv={deriv} n={n} sigma={sigma}: {e:.2e}")
            assert e < 1e-4, (n, sigma, e)
        off += n


@pytest.mark.parametrize("K,norm", [(3, 0), (4, 0), (6, 0), (3, 1), (4, 1)])
def test_multiply_method(K, norm):
    """The multiplication method (Sec. III-B: 2K - 1 non-harmonic window sums, complex combine; with
    norm = 1 also the K harmonic kappa terms of the normalised Morlet) on a ragged batch against the
    direct convolution with the oracle's own kernel; FP32 recursion, gate 1e-4 of max|W| like the
    other uncompensated form. Windows beyond L = 4096 (sigma 2000 and 3000) start from window sums of
    tile sums."""
    import torch
    rng = np.random.default_rng(40 + K + 10 * norm)
    lens = [30000, 7, 4097, 12000, 70001]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    xi = 6.0 if norm == 0 else 2.0  # kappa_xi = e^{-2}: the kappa terms matter
    sigmas = [8.0, 40.0, 300.0, 1000.0, 2000.0, 3000.0]
    plan = m.morlet_plan(lens, sigmas, K=K, xi=xi, method=m.MORLET_MULTIPLY, precision=m.MORLET_FP32_PLAIN,
                         norm=norm)
    st = m.morlet_plan_stats(plan)
    assert st["rows_lookback"] == 0 and st["rows_start_state"] == 2 * len(lens), st
    S, n_in = len(sigmas), sum(lens)
    xt = torch.from_numpy(np.concatenate(sigs)).cuda()
    W = torch.full((n_in * S,), float("nan"), dtype=torch.complex64, device="cuda")
    m.morlet_forward(plan, xt, W)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    Wh = W.cpu().numpy()
    refs = [[om.morlet_multiply_direct(x.astype(np.float64), om.fit_multiply(sigma, xi, K, norm=norm))
             for sigma in sigmas] for x in sigs]
    off = 0
    for i, n in enumerate(lens):
        for s, sigma in enumerate(sigmas):
            got = Wh[S * off + s * n: S * off + (s + 1) * n]
            e = rel_err(got, refs[i][s])
            print(f"multiply K={K} norm={norm} n={n} sigma={sigma}: {e:.2e}")
            assert e < 1e-4, (n, sigma, e)
        off += n
    # Horner start states from shorter windows on (every row at 1), longest items first
    for h in (512, 1):
        m.morlet_plan_set_row_thresholds(plan, 0, h)
        m.morlet_plan_set_schedule(plan, 16, 64, 2, 0)
        st = m.morlet_plan_stats(plan)
        assert st["rows_start_state"] == sum(4 * sg > h for sg in sigmas) * len(lens), (h, st)
        W = torch.full((n_in * S,), float("nan"), dtype=torch.complex64, device="cuda")
        m.morlet_forward(plan, xt, W)
        torch.cuda.synchronize()
        assert m.morlet_last_device_error(plan) == 0
        Wh = W.cpu().numpy()
        off = 0
        for i, n in enumerate(lens):
            for s, sigma in enumerate(sigmas):
                e = rel_err(Wh[S * off + s * n: S * off + (s + 1) * n], refs[i][s])
                assert e < 1e-4, (h, n, sigma, e)
            off += n


@pytest.mark.parametrize("sigma,tail", [(300.0, 1 << 17), (2000.0, 1 << 17), (10321.27, 1 << 15)])
def test_multiply_method_long_signal(sigma, tail):
    """The multiplication method's non-harmonic powers e^{i omega0 n} are formed from an FP64 angle
    (reduced mod 2 pi) times an exact harmonic: on a 2^24-sample signal (window segments at sigma 300,
    start-state items at 2000 and at the c3 scalogram's largest scale, L = 41286) outputs up to
    n = 2^24 - 1 agree with the direct sum of the oracle's kernel, at sampled n everywhere in the row
    and on a full stretch at its end."""
    import torch
    N, K = 1 << 24, 4
    x = WL.c5_pink()
    mf = om.fit_multiply(sigma, 6.0, K)
    plan = m.morlet_plan([N], [sigma], K=K, method=m.MORLET_MULTIPLY, precision=m.MORLET_FP32_PLAIN)
    W = torch.empty(N, dtype=torch.complex64, device="cuda")
    m.morlet_forward(plan, torch.from_numpy(x).cuda(), W)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    rng = np.random.default_rng(int(sigma))
    idx = np.unique(np.concatenate([[0, 1, N // 2, N - 2, N - 1], rng.integers(0, N, 64)]))
    ref = om.morlet_multiply_direct(x.astype(np.float64), mf, idx)
    M = tail + 2 * mf["L"]
    ref_tail = om.morlet_multiply_direct(x[N - M:].astype(np.float64), mf)[M - tail:]
    Wh = W.cpu().numpy()
    scale = np.abs(ref_tail).max()
    e_s = float(np.abs(Wh[idx] - ref).max() / scale)
    e_t = float(np.abs(Wh[N - tail:] - ref_tail).max() / scale)
    print(f"multiply N=2^24 sigma={sigma}: sampled {e_s:.2e}, last {tail} outputs {e_t:.2e}")
    assert e_s < 1e-4 and e_t < 1e-4


@pytest.mark.parametrize("precision", [m.MORLET_FP32_COMP, m.MORLET_FP64])
def test_gauss_filter_2d(precision):
    """Separable 2-D Gaussian filtering (rows, transpose, columns, transpose back) against the
    oracle's separable reference: an odd-sized image, several scales and derivative pairs; a
    second call with the same key reuses the cached plans and workspace."""
    import torch
    rng = np.random.default_rng(60)
    ny, nx = 301, 517
    img = rng.standard_normal((ny, nx))
    f64 = precision == m.MORLET_FP64
    dt = torch.float64 if f64 else torch.float32
    xin = img if f64 else img.astype(np.float32).astype(np.float64)
    it = torch.from_numpy(xin).to(dt).cuda().contiguous()
    for sigma, P, dy, dx in ((2.5, 4, 0, 0), (12.0, 6, 1, 0), (7.0, 6, 0, 2), (30.0, 5, 2, 1)):
        out = torch.full((ny, nx), float("nan"), dtype=dt, device="cuda")
        for _ in range(2):
            m.gauss_filter_2d(it, ny, nx, sigma, P, dy, dx, precision, out)
        torch.cuda.synchronize()
        ref = om.gauss_filter_2d_direct(xin, sigma, P, dy, dx)
        e = rel_err(out.cpu().numpy(), ref)
        print(f"gauss 2d sigma={sigma} P={P} dy={dy} dx={dx} precision={precision}: {e:.2e}")
        assert e < (1e-12 if f64 else 1e-5), (sigma, dy, dx, e)


@pytest.mark.parametrize("case", ["comp", "fp64", "asft", "gauss_d1"])
def test_edge_extension(case):
    """MORLET_FLAG_EDGE: every row kind (lane chunks, window segments, start-state items; look-back
    chains in FP64) on ragged signals, some shorter than the window, against the oracle run on the
    edge-padded signal; nothing is written outside the scalogram."""
    import torch
    rng = np.random.default_rng(70)
    lens = [1, 5, 1000, 30000, 70001]
    sigs = [rng.standard_normal(n) for n in lens]
    K = 4
    if case == "gauss_d1":
        sigmas, P = [5.0, 40.0, 700.0, 3000.0], 6
        kw = dict(K=P + 1, method=m.MORLET_GAUSS, deriv=1, precision=m.MORLET_FP32_COMP)
    elif case == "asft":
        sigmas = [8.0, 40.0, 300.0]
        kw = dict(K=K, transform=m.MORLET_ASFT, precision=m.MORLET_FP32_PLAIN)
    else:
        sigmas = [8.0, 40.0, 700.0, 3000.0]
        kw = dict(K=K, precision=m.MORLET_FP64 if case == "fp64" else m.MORLET_FP32_COMP)
    f64 = kw["precision"] == m.MORLET_FP64
    real = case == "gauss_d1"
    plan = m.morlet_plan(lens, sigmas, flags=m.MORLET_FLAG_EDGE, **kw)
    S, n_in = len(sigmas), sum(lens)
    xs = [v if f64 else v.astype(np.float32) for v in sigs]
    xt = torch.from_numpy(np.concatenate(xs)).cuda()
    dt = (torch.float64 if f64 else torch.float32) if real else (torch.complex128 if f64 else torch.complex64)
    W = torch.full((n_in * S + 8,), float("nan"), dtype=dt, device="cuda")
    m.morlet_forward(plan, xt, W)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    Wh = W.cpu().numpy()
    assert np.all(np.isnan(Wh[n_in * S:].real))
    # Rows shorter than the window are nearly constant once extended by their edge values, and the
    # transform of a constant nearly cancels (the wavelet's mean is small): their error is measured
    # against sum|kernel| max|x|, the scale of the arithmetic's rounding, instead of max|W|.
    tol = {"comp": 1e-5, "fp64": 1e-12, "asft": 1e-4, "gauss_d1": 1e-5}[case]
    bad = []
    off = 0
    for x, n in zip(xs, lens):
        xd = x.astype(np.float64)
        for s, sg in enumerate(sigmas):
            if real:
                gf = om.fit_gauss(sg, P, 1)
                E = gf["L"]
                ref = sft_dd.sft_gauss(om.edge_extended(xd, E), gf)[E:E + n]
                knorm = np.abs(om.kernel_gauss(gf)).sum()
            elif case == "asft":
                E = om.window_half(sg) + om.default_n0(sg)
                ref = oracle_forward(om.edge_extended(xd, E), sg, K, transform=m.MORLET_ASFT)[E:E + n]
                knorm = np.abs(om.kernel_asft(om.fit_direct(sg, 6.0, K), sg, 6.0, om.default_n0(sg))[1]).sum()
            else:
                E = om.window_half(sg)
                ref = oracle_forward(om.edge_extended(xd, E), sg, K)[E:E + n]
                knorm = np.abs(om.kernel_direct(om.fit_direct(sg, 6.0, K))).sum()
            got = Wh[S * off + s * n: S * off + (s + 1) * n]
            scale = np.abs(ref).max()
            if n < 2 * om.window_half(sg):
                scale = max(scale, knorm * np.abs(xd).max())
            e = float(np.abs(got - ref).max() / scale)
            if not e < tol:
                bad.append((n, sg, e))
        off += n
    assert not bad, (case, bad)
    with pytest.raises(m.MorletError) as err:
        g = torch.zeros(n_in * S, dtype=dt, device="cuda")
        m.morlet_backward(plan, g, torch.zeros(n_in, dtype=torch.float64 if f64 else torch.float32, device="cuda"))
    assert err.value.code == m.MORLET_ERR_UNSUPPORTED
