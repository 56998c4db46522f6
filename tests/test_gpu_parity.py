"""GPU parity: the CUDA library through its C ABI against the CPU oracle on the same seeded inputs.

Tolerances (relative max-abs error over max |W| of the oracle):
  compensated FP32 (FP32 scan, two-float carries and prefix sums): 1e-5;  FP64: 1e-12;
  plain FP32 and ASFT FP32: reported by print, gated only loosely (1e-3 / 1e-4) since the method's
  plain-FP32 error grows with the row length.
"""
import math

import numpy as np
import pytest

import paper_2110_11866_gb300 as m
import workloads as WL
from oracle import morlet as om
from oracle import sft_dd
from tests.gpu_helpers import gpu_forward, oracle_forward, rel_err

pytestmark = pytest.mark.gpu

TOL = {m.MORLET_FP32_COMP: 1e-5, m.MORLET_FP64: 1e-12, m.MORLET_FP32_PLAIN: 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("form", [m.MORLET_FORM_ROTATING, m.MORLET_FORM_KERNEL])
def test_c1_fp64_single_signal(form):
    """Config 1: N = 4096 N(0,1) float64, sigma = 64, K = 4, FP64 path vs the double-double oracle."""
    w = WL.c1_fp64_single()
    x = w.signals[0]
    plan, out = gpu_forward([x], [64.0], K=4, precision=m.MORLET_FP64, form=form)
    ref = oracle_forward(x, 64.0, 4)
    e = rel_err(out[0][0], ref)
    print(f"c1 fp64 form={form} rel err {e:.3e}")
    assert e < 1e-12
    # the fit: same harmonics and coefficients as the oracle's independent FP64 least squares
    info = m.morlet_plan_info(plan, 0)
    fit = om.fit_direct(64.0, 6.0, 4)
    assert info["p0"] == fit["p0"] and info["L"] == fit["L"] == 256
    assert np.abs(np.array(info["m"]) - fit["m"]).max() < 1e-12
    assert np.abs(np.array(info["l"]) - fit["l"]).max() < 1e-12
    # approximation error of the method itself (reported, K = 4, L = 4 sigma)
    true = om.morlet_true_direct(x, 64.0, 6.0)
    print(f"c1 SFT vs direct +-8 sigma Morlet: {rel_err(ref, true):.3e}")


@pytest.mark.parametrize("K", [2, 4, 6])
@pytest.mark.parametrize("shift", [0, 1, 3])
def test_lane_chunk_rows_and_unaligned_buffers(K, shift):
    """Short windows in compensated FP32 go through the lane-chunk scan: rows shorter than a lane
    chunk, rows spanning several work items, odd and even output offsets, both parities of L, and
    input / output buffers that start `shift` elements past a 16-byte boundary."""
    import torch
    rng = np.random.default_rng(500 + 10 * K + shift)
    lens = [1, 5, 17, 1000, 33333, 70001, 4096]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    sigmas = [8.0, 13.25, 32.0, 64.0]   # L = 32, 53, 128 in lane chunks; L = 256 in window segments
    plan = m.morlet_plan(lens, sigmas, K=K, precision=m.MORLET_FP32_COMP)
    st = m.morlet_plan_stats(plan)
    assert st["rows_lane_chunk"] == len(lens) * 3 and st["lane_chunk_items"] > 0
    S, n_in = len(sigmas), sum(lens)
    xb = torch.zeros(n_in + 4, dtype=torch.float32, device="cuda")
    xb[shift:shift + n_in] = torch.from_numpy(np.concatenate(sigs)).cuda()
    Wb = torch.zeros(n_in * S + 4, dtype=torch.complex64, device="cuda")
    m.morlet_forward(plan, xb[shift:], Wb[shift:])
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    Wh = Wb.cpu().numpy()
    assert np.all(Wh[:shift] == 0) and np.all(Wh[shift + n_in * S:] == 0)  # nothing written outside
    off = 0
    for x, n in zip(sigs, lens):
        for s, sg in enumerate(sigmas):
            got = Wh[shift + S * off + s * n: shift + S * off + (s + 1) * n]
            e = rel_err(got, oracle_forward(x.astype(np.float64), sg, K))
            assert e < 1e-5, (n, sg, e)
        off += n


@pytest.mark.parametrize("K", [3, 4, 6])
@pytest.mark.parametrize("longest", [4000.0, 9000.0])
def test_start_state_rows(K, longest):
    """Long windows in compensated FP32: work items start from exact states (several chunks per row,
    every input alignment mod 16 bytes, rows shorter than a tile, shorter than the window, and rows
    spanning many work items), next to short-window rows of the same plan. With the longest sigma
    4000 the states are window sums of tile sums; with 9000 (windows of 141 tiles against items of
    4 tiles) they come from the chained prefix sums."""
    rng = np.random.default_rng(300 + K)
    lens = [100000, 3, 50001, 262149, 1030, 77777]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    sigmas = [20.0, 255.0, 1030.0, 2000.0, longest]
    plan, out = gpu_forward(sigs, sigmas, K=K, precision=m.MORLET_FP32_COMP)
    st = m.morlet_plan_stats(plan)
    assert st["rows_start_state"] == len(lens) * 3 and st["prefix_items"] > 0
    assert st["start_state_window_sums"] == (1 if longest < 5000 else 0)
    worst = 0.0
    for i, x in enumerate(sigs):
        for s, sg in enumerate(sigmas):
            ref = oracle_forward(x.astype(np.float64), sg, K)
            e = rel_err(out[i][s], ref)
            worst = max(worst, e)
            assert e < 1e-5, (i, sg, e)
    print(f"start-state rows K={K}: worst {worst:.3e}")


@pytest.mark.parametrize("K", [3, 4, 6])
def test_asft_start_state_rows(K):
    """The ASFT's long windows (L > 4096) start from window sums of damped FP32 tile sums (Horner lane
    sums, 2L + 1 samples): rows shorter than a tile, shorter than the window, spanning many work
    items, every input alignment, next to window-segment rows of the same plan; the Morlet and the
    Gaussian first derivative (real output), each against the oracle's double-double recursion."""
    rng = np.random.default_rng(700 + K)
    lens = [100000, 3, 50001, 262149, 1030, 77777]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    sigmas = [20.0, 800.0, 2000.0, 5000.0]  # L = 80, 3200 (window segments), 8000, 20000 (start states)
    plan, out = gpu_forward(sigs, sigmas, K=K, precision=m.MORLET_FP32_PLAIN, transform=m.MORLET_ASFT)
    st = m.morlet_plan_stats(plan)
    assert st["rows_start_state"] == 2 * len(lens) and st["rows_lookback"] == 0, st
    worst = 0.0
    for i, x in enumerate(sigs):
        for s, sg in enumerate(sigmas):
            e = rel_err(out[i][s], oracle_forward(x.astype(np.float64), sg, K, transform=m.MORLET_ASFT))
            worst = max(worst, e)
            assert e < 1e-4, (i, sg, e)
    print(f"ASFT start-state rows K={K}: worst {worst:.2e}")
    # Horner start states from shorter windows on, down to every row, in both item orders
    import torch
    refs = [[oracle_forward(x.astype(np.float64), sg, K, transform=m.MORLET_ASFT) for sg in sigmas] for x in sigs]
    xt = torch.from_numpy(np.concatenate(sigs)).cuda()
    S, n_in = len(sigmas), sum(lens)
    for h in (512, 1):
        for order in (0, 2):
            m.morlet_plan_set_row_thresholds(plan, 0, h)
            m.morlet_plan_set_schedule(plan, 16, 64, order, 0)
            st = m.morlet_plan_stats(plan)
            assert st["rows_start_state"] == sum(4 * sg > h for sg in sigmas) * len(lens), (h, st)
            assert m.morlet_plan_schedule(plan)["start_state_min_L"] == h
            W = torch.full((n_in * S,), float("nan"), dtype=torch.complex64, device="cuda")
            m.morlet_forward(plan, xt, W)
            torch.cuda.synchronize()
            assert m.morlet_last_device_error(plan) == 0
            Wh = W.cpu().numpy()
            off = 0
            for i, n in enumerate(lens):
                for s, sg in enumerate(sigmas):
                    e = rel_err(Wh[S * off + s * n: S * off + (s + 1) * n], refs[i][s])
                    assert e < 1e-4, (h, order, i, sg, e)
                off += n
    with pytest.raises(m.MorletError):
        m.morlet_plan_set_row_thresholds(plan, 0, 4097)
    import torch
    P = K + 3
    gplan = m.morlet_plan(lens, sigmas, K=P + 1, method=m.MORLET_GAUSS, transform=m.MORLET_ASFT, deriv=1,
                          precision=m.MORLET_FP32_PLAIN)
    assert m.morlet_plan_stats(gplan)["rows_start_state"] == 2 * len(lens)
    S, n_in = len(sigmas), sum(lens)
    y = torch.full((n_in * S,), float("nan"), dtype=torch.float32, device="cuda")
    m.morlet_forward(gplan, torch.from_numpy(np.concatenate(sigs)).cuda(), y)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(gplan) == 0
    yh = y.cpu().numpy()
    # A row shorter than the window gives a derivative that nearly cancels (the kernel is odd): its
    # error is measured against sum|kernel| max|x|, the scale of the arithmetic's rounding.
    off = 0
    for x, n in zip(sigs, lens):
        for s, sg in enumerate(sigmas):
            gf = om.fit_gauss_asft(sg, P, 1, om.default_n0(sg))
            ref = sft_dd.asft_gauss(x.astype(np.float64), gf)
            scale = np.abs(ref).max()
            if n < 2 * gf["L"]:
                scale = max(scale, np.abs(om.kernel_gauss_asft(gf)[1]).sum() * np.abs(x).max())
            e = float(np.abs(yh[S * off + s * n: S * off + (s + 1) * n] - ref).max() / scale)
            assert e < 1e-4, (n, sg, e)
        off += n


@pytest.mark.parametrize("precision", [m.MORLET_FP32_COMP, m.MORLET_FP32_PLAIN, m.MORLET_FP64])
@pytest.mark.parametrize("form", [m.MORLET_FORM_ROTATING, m.MORLET_FORM_KERNEL])
@pytest.mark.parametrize("K", [2, 3, 4, 5, 6, 8, 12])
def test_small_shapes(precision, form, K):
    """Ragged lengths that straddle tile edges (4096 outputs per sub-tile) and short windows."""
    rng = np.random.default_rng(100 + K)
    lens = [1, 7, 4095, 4096, 4097, 9000, 20000]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    sigmas = [8.0, 37.5, 300.0, 1500.0]
    plan, out = gpu_forward(sigs, sigmas, K=K, precision=precision, form=form)
    worst = 0.0
    for i, x in enumerate(sigs):
        for s, sg in enumerate(sigmas):
            ref = oracle_forward(x, sg, K)
            worst = max(worst, rel_err(out[i][s], ref))
    print(f"K={K} precision={precision} form={form} worst rel err {worst:.3e}")
    assert worst < TOL[precision]


def test_n_shorter_than_window():
    """Signals far shorter than the window (L >> N): outputs still equal the zero-extended sums."""
    rng = np.random.default_rng(5)
    sigs = [rng.standard_normal(n).astype(np.float32) for n in (3, 100, 1000)]
    plan, out = gpu_forward(sigs, [2000.0, 10321.0], K=4)
    for i, x in enumerate(sigs):
        for s, sg in enumerate([2000.0, 10321.0]):
            assert rel_err(out[i][s], oracle_forward(x, sg, 4)) < 1e-5


@pytest.mark.parametrize("sigma", WL.C2_SIGMAS)
@pytest.mark.parametrize("K", WL.C2_KS)
def test_c2_chirps_forms(sigma, K):
    """Config 2: N = 102400 chirps + noise, sigma sweep x K x {plain, compensated, ASFT} FP32."""
    x = WL.c2_chirps()
    ref = oracle_forward(x, sigma, K)
    _, comp = gpu_forward([x], [sigma], K=K, precision=m.MORLET_FP32_COMP)
    _, plain = gpu_forward([x], [sigma], K=K, precision=m.MORLET_FP32_PLAIN)
    _, ki = gpu_forward([x], [sigma], K=K, precision=m.MORLET_FP32_COMP, form=m.MORLET_FORM_KERNEL)
    ea = rel_err(comp[0][0], ref)
    ep = rel_err(plain[0][0], ref)
    ek = rel_err(ki[0][0], ref)
    refa = oracle_forward(x, sigma, K, transform=m.MORLET_ASFT)
    _, asft = gpu_forward([x], [sigma], K=K, precision=m.MORLET_FP32_PLAIN, transform=m.MORLET_ASFT)
    es = rel_err(asft[0][0], refa)
    print(f"c2 sigma={sigma} K={K}: comp {ea:.2e} kernel-integral {ek:.2e} plain {ep:.2e} asft {es:.2e}")
    assert ea < 1e-5 and ek < 1e-5
    assert ep < 1e-3
    assert es < 1e-4


def test_autotune_keeps_results():
    """MORLET_FLAG_AUTOTUNE picks row thresholds by timing; whatever it picks, the transform is the
    same to within the compensated-FP32 gate."""
    rng = np.random.default_rng(77)
    lens = [50000, 120000, 3000]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    sigmas = [8.0, 40.0, 300.0, 1500.0]
    plan, out = gpu_forward(sigs, sigmas, K=4, flags=m.MORLET_FLAG_AUTOTUNE)
    st = m.morlet_plan_stats(plan)
    pairs = [(128, 2048), (256, 2048), (64, 2048), (0, 2048), (128, 1024), (256, 1024), (64, 1024), (0, 1024),
             (128, 512), (256, 512), (128, 128), (64, 64), (0, 1)]
    assert (st["lane_chunk_max_L"], st["start_state_min_L"]) in pairs, st
    sc = m.morlet_plan_schedule(plan)
    assert sc["autotuned"] == 1 and sc["autotune_outputs"] == sum(lens) * len(sigmas), sc
    assert sc["seg_mult"] in (8, 12, 16) and sc["ss_tiles_max"] in (16, 32, 64) and sc["order"] in (0, 1, 2)
    for i, x in enumerate(sigs):
        for s, sg in enumerate(sigmas):
            assert rel_err(out[i][s], oracle_forward(x.astype(np.float64), sg, 4)) < 1e-5


@pytest.mark.parametrize("K", [3, 6])
def test_every_autotune_choice_passes(K):
    """Each (lane-chunk, start-state) threshold pair the autotuner may keep gives the transform within
    the compensated-FP32 gate, on rows that move between the scans as the thresholds change
    (L = 32 ... 4800), for white noise and for a chirp through the kernels' bands (the resonant
    worst case); pairs outside the accepted ranges are refused."""
    import torch
    rng = np.random.default_rng(900 + K)
    sigs = [rng.standard_normal(n).astype(np.float32) for n in (70001, 3000, 150000)]
    sigs.append(WL.c2_chirps().astype(np.float32))
    lens = [len(x) for x in sigs]
    sigmas = [8.0, 16.0, 40.0, 64.0, 100.0, 300.0, 600.0, 1200.0]
    refs = [[oracle_forward(x.astype(np.float64), sg, K) for sg in sigmas] for x in sigs]
    plan = m.morlet_plan(lens, sigmas, K=K, precision=m.MORLET_FP32_COMP)
    S, n_in = len(sigmas), sum(lens)
    xt = torch.from_numpy(np.concatenate(sigs)).cuda()
    for bad in [(128, 4096), (128, 0), (512, 2048), (-1, 2048)]:
        with pytest.raises(m.MorletError) as err:
            m.morlet_plan_set_row_thresholds(plan, *bad)
        assert err.value.code == m.MORLET_ERR_ARG
    pairs = [(128, 2048), (256, 2048), (64, 2048), (0, 2048), (128, 1024), (256, 1024), (64, 1024), (0, 1024),
             (128, 512), (256, 512), (128, 128), (64, 64), (0, 1)]
    for ls, ss in pairs:
        m.morlet_plan_set_row_thresholds(plan, ls, ss)
        st = m.morlet_plan_stats(plan)
        assert (st["lane_chunk_max_L"], st["start_state_min_L"]) == (ls, ss)
        n_lane = sum(int(np.ceil(4 * sg)) <= ls for sg in sigmas) * len(lens)
        assert st["rows_lane_chunk"] == n_lane, (ls, ss, st)
        W = torch.full((n_in * S,), float("nan"), dtype=torch.complex64, device="cuda")
        m.morlet_forward(plan, xt, W)
        torch.cuda.synchronize()
        assert m.morlet_last_device_error(plan) == 0
        Wh = W.cpu().numpy()
        off = 0
        for i, n in enumerate(lens):
            for s in range(S):
                got = Wh[S * off + s * n: S * off + (s + 1) * n]
                e = rel_err(got, refs[i][s])
                assert e < 1e-5, (ls, ss, n, sigmas[s], e)
            off += n


@pytest.mark.parametrize("K", [3, 4, 6])
def test_chirp_sigma_sweep(K):
    """A linear chirp through the kernels' bands (the resonant worst case for the FP32 recursions)
    at every row kind of the default schedule: lane chunks, window segments up to L = 2048, and
    start-state items beyond (window sums of tile sums for the shorter windows, prefix sums for
    the longest)."""
    x = WL.c2_chirps().astype(np.float32)
    for sigmas, window_sums in (([8.0, 32.0, 64.0, 128.0, 362.0, 512.0, 724.0, 1024.0, 1448.0, 2048.0, 2896.0], 1),
                                ([4096.0, 5793.0, 8192.0, 10321.0], 0)):
        plan, out = gpu_forward([x], sigmas, K=K)
        assert m.morlet_plan_stats(plan)["start_state_window_sums"] == window_sums
        for s, sg in enumerate(sigmas):
            e = rel_err(out[0][s], oracle_forward(x.astype(np.float64), sg, K))
            assert e < 1e-5, (sg, K, e)


@pytest.mark.parametrize("K", [3, 4, 6])
@pytest.mark.parametrize("ls,ss,seed", [(0, 1, 1), (64, 64, 1), (128, 128, 1), (0, 1, 11), (0, 1, 13)])
def test_chirp_sigma_sweep_start_state_everywhere(K, ls, ss, seed):
    """The chirp through the kernels' bands (several seeds of the recipe) with start-state items for
    every row above the lane-chunk limit (no window segments), items of the longest accepted length
    (64 tiles), in both item orders: start states from window sums of tile sums at every window
    length."""
    x = WL.c2_chirps(seed).astype(np.float32)
    sigmas = [8.0, 11.0, 16.0, 32.0, 64.0, 128.0, 362.0, 1024.0, 2896.0]
    refs = [oracle_forward(x.astype(np.float64), sg, K) for sg in sigmas]
    import torch
    plan = m.morlet_plan([len(x)], sigmas, K=K, precision=m.MORLET_FP32_COMP)
    xt = torch.from_numpy(x).cuda()
    for order in (0, 2):
        m.morlet_plan_set_row_thresholds(plan, ls, ss)
        m.morlet_plan_set_schedule(plan, 16, 64, order, 0)
        st = m.morlet_plan_stats(plan)
        n_lane = sum(int(np.ceil(4 * sg)) <= ls for sg in sigmas)
        assert st["rows_lane_chunk"] == n_lane and st["rows_start_state"] == len(sigmas) - n_lane, st
        W = torch.full((len(x) * len(sigmas),), float("nan"), dtype=torch.complex64, device="cuda")
        m.morlet_forward(plan, xt, W)
        torch.cuda.synchronize()
        assert m.morlet_last_device_error(plan) == 0
        Wh = W.cpu().numpy().reshape(len(sigmas), len(x))
        for s, sg in enumerate(sigmas):
            e = rel_err(Wh[s], refs[s])
            assert e < 1e-5, (ls, ss, order, sg, K, e)


@pytest.mark.parametrize("K", [4, 6])
def test_chirp_sigma_sweep_other_forms(K):
    """The chirp sweep for the kernel-integral form (compensated FP32), plain FP32, FP64 and the
    ASFT, each against its own gate."""
    x = WL.c2_chirps()
    sigmas = [128.0, 512.0, 1024.0, 2048.0, 2896.0, 4096.0, 10321.0]
    refs = [oracle_forward(x, sg, K) for sg in sigmas]
    cases = [(dict(precision=m.MORLET_FP32_COMP, form=m.MORLET_FORM_KERNEL), refs, 1e-5),
             (dict(precision=m.MORLET_FP32_PLAIN), refs, 1e-3),
             (dict(precision=m.MORLET_FP64), refs, 1e-12),
             (dict(precision=m.MORLET_FP32_PLAIN, transform=m.MORLET_ASFT),
              [oracle_forward(x, sg, K, transform=m.MORLET_ASFT) for sg in sigmas], 1e-4)]
    for kw, rr, tol in cases:
        _, out = gpu_forward([x], sigmas, K=K, **kw)
        for s, sg in enumerate(sigmas):
            e = rel_err(out[0][s], rr[s])
            assert e < tol, (kw, sg, e)


def test_chirp_long_windows_from_tile_sums():
    """Window sums of tile sums at the longest windows (a batch large enough that start-state items
    are long, so the plan takes window sums): the chirp stays within the gate."""
    import torch
    base = WL.c2_chirps().astype(np.float32)
    rng = np.random.default_rng(11)
    sigs = [np.roll(base, int(rng.integers(len(base)))) for _ in range(256)]
    lens = [len(v) for v in sigs]
    sigmas = [4096.0, 5793.0, 8192.0, 10321.0]
    K = 6
    plan = m.morlet_plan(lens, sigmas, K=K, precision=m.MORLET_FP32_COMP)
    assert m.morlet_plan_stats(plan)["start_state_window_sums"] == 1
    xt = torch.from_numpy(np.concatenate(sigs)).cuda()
    W = torch.empty(sum(lens) * len(sigmas), dtype=torch.complex64, device="cuda")
    m.morlet_forward(plan, xt, W)
    torch.cuda.synchronize()
    assert m.morlet_last_device_error(plan) == 0
    S = len(sigmas)
    for i in (0, 97, 255):
        row = S * sum(lens[:i])
        for s, sg in enumerate(sigmas):
            got = W[row + s * lens[i]: row + (s + 1) * lens[i]].cpu().numpy()
            e = rel_err(got, oracle_forward(sigs[i].astype(np.float64), sg, K))
            assert e < 1e-5, (i, sg, e)


@pytest.mark.parametrize("seed", [1, 11, 12, 13])
def test_chirp_seeds_default_schedule(seed):
    """Config 2's chirp recipe (three linear chirps in 0.001-0.2 rad/sample plus N(0, 0.1^2)) drawn
    from several seeds, at all six of its scales and K = 4 and 6, through the default compensated
    schedule (lane chunks, window segments, start-state items): every row within 1e-5 of the
    oracle's max |W|. The chirps sweep through the kernels' bands, the resonant worst case of the FP32
    recursions."""
    x = WL.c2_chirps(seed)
    worst = {}
    for K in (4, 6):
        _, out = gpu_forward([x], WL.C2_SIGMAS, K=K, precision=m.MORLET_FP32_COMP)
        for s, sg in enumerate(WL.C2_SIGMAS):
            e = rel_err(out[0][s], oracle_forward(x.astype(np.float64), sg, K))
            worst[(sg, K)] = e
    print(f"chirp seed {seed}: " + ", ".join(f"sigma {sg:g} K {K}: {e:.2e}" for (sg, K), e in worst.items()))
    bad = {k: v for k, v in worst.items() if not v < 1e-5}
    assert not bad, bad


SCHEDULES = [(16, 32, 0), (12, 32, 0), (8, 32, 0), (16, 16, 1), (16, 64, 1), (8, 64, 1), (16, 32, 2), (8, 16, 2)]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_every_schedule_passes(sched):
    """Every schedule the autotuner may pick (window-segment length, start-state item size, scale
    order) gives the transform within the compensated-FP32 gate, on white noise and on a chirp through
    the kernels' bands, at windows in every row kind (L = 32 ... 8192); the ASFT likewise with one
    chain per row or window segments, within its gate."""
    import torch
    seg_mult, ss_tiles, order = sched
    rng = np.random.default_rng(1000 + seg_mult + ss_tiles + order)
    sigs = [rng.standard_normal(n).astype(np.float32) for n in (70001, 3000, 150000)]
    sigs.append(WL.c2_chirps(12).astype(np.float32))
    lens = [len(v) for v in sigs]
    sigmas = [8.0, 40.0, 300.0, 512.0, 1024.0, 2048.0]
    S, n_in = len(sigmas), sum(lens)
    xt = torch.from_numpy(np.concatenate(sigs)).cuda()
    for K, kw, tol, fn in ((6, dict(precision=m.MORLET_FP32_COMP), 1e-5, m.MORLET_SFT),
                           (4, dict(precision=m.MORLET_FP32_PLAIN, transform=m.MORLET_ASFT), 1e-4, m.MORLET_ASFT)):
        plan = m.morlet_plan(lens, sigmas, K=K, **kw)
        for chains in ((0, 1) if fn == m.MORLET_ASFT else (0,)):
            m.morlet_plan_set_schedule(plan, seg_mult, ss_tiles, order, chains)
            sc = m.morlet_plan_schedule(plan)
            assert (sc["seg_mult"], sc["ss_tiles_max"], sc["order"], sc["asft_chains"]) == (seg_mult, ss_tiles, order, chains)
            W = torch.full((n_in * S,), float("nan"), dtype=torch.complex64, device="cuda")
            m.morlet_forward(plan, xt, W)
            torch.cuda.synchronize()
            assert m.morlet_last_device_error(plan) == 0
            Wh = W.cpu().numpy()
            off = 0
            for i, n in enumerate(lens):
                for s, sg in enumerate(sigmas):
                    got = Wh[S * off + s * n: S * off + (s + 1) * n]
                    e = rel_err(got, oracle_forward(sigs[i].astype(np.float64), sg, K, transform=fn))
                    assert e < tol, (sched, fn, chains, n, sg, e)
                off += n
    with pytest.raises(m.MorletError) as err:
        m.morlet_plan_set_schedule(plan, 24, 32, 0, 0)
    assert err.value.code == m.MORLET_ERR_ARG


def test_autotune_times_a_bounded_subset_when_memory_is_short():
    """The autotuner times the whole batch when its scratch copy takes at most a quarter of the free
    device memory, and otherwise a sub-plan of every k-th signal holding at most 2^28 outputs (no
    full-size scratch scalogram); the plan reports which. Memory is made short by holding most of
    the free memory in a torch buffer while the plan is built."""
    import torch
    lens = [1 << 20] * 300  # 629 M outputs at two scales: 5 GB of scratch output
    plan = m.morlet_plan(lens, [8.0, 300.0], K=4, flags=m.MORLET_FLAG_AUTOTUNE)
    sc = m.morlet_plan_schedule(plan)
    assert sc["autotuned"] == 1 and sc["autotune_outputs"] == 2 * sum(lens), sc
    del plan
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    hold = torch.empty(int(free - (12 << 30)), dtype=torch.uint8, device="cuda")  # leave 12 GB free
    try:
        plan = m.morlet_plan(lens, [8.0, 300.0], K=4, flags=m.MORLET_FLAG_AUTOTUNE)
        sc = m.morlet_plan_schedule(plan)
        assert sc["autotuned"] == 1 and 0 < sc["autotune_outputs"] <= (1 << 28) < 2 * sum(lens), sc
        del plan
    finally:
        del hold
        torch.cuda.empty_cache()


def test_autotune_asft_keeps_results():
    """MORLET_FLAG_AUTOTUNE on an ASFT plan chooses between window segments and one chain per row
    (and the segment length) by timing; the transform stays within the ASFT gate."""
    rng = np.random.default_rng(78)
    lens = [50000, 120000, 3000]
    sigs = [rng.standard_normal(n).astype(np.float32) for n in lens]
    sigmas = [8.0, 300.0, 1500.0]
    plan, out = gpu_forward(sigs, sigmas, K=4, precision=m.MORLET_FP32_PLAIN, transform=m.MORLET_ASFT,
                            flags=m.MORLET_FLAG_AUTOTUNE)
    sc = m.morlet_plan_schedule(plan)
    assert sc["autotuned"] == 1 and sc["asft_chains"] in (0, 1), sc
    for i, x in enumerate(sigs):
        for s, sg in enumerate(sigmas):
            ref = oracle_forward(x.astype(np.float64), sg, 4, transform=m.MORLET_ASFT)
            assert rel_err(out[i][s], ref) < 1e-4


def test_fp64_rate_measurement():
    """The FP64 FMA rate helper returns a plausible rate for this GPU (between 0.1 and 100 TFLOP/s)."""
    r = m.morlet_measure_fp64_rate()
    print(f"measured FP64 FMA rate: {r / 1e12:.3f} TFLOP/s")
    assert 1e11 < r < 1e14


def test_deterministic_replay():
    """Two launches (graph replays) give bit-identical outputs."""
    x = WL.white(3, 300000)
    import torch
    plan = m.morlet_plan([len(x)], [12.0, 900.0, 5000.0], K=4)
    xt = torch.from_numpy(x).cuda()
    W1 = torch.empty(len(x) * 3, dtype=torch.complex64, device="cuda")
    W2 = torch.empty_like(W1)
    m.morlet_forward(plan, xt, W1)
    m.morlet_forward(plan, xt, W2)
    torch.cuda.synchronize()
    assert torch.equal(W1, W2)


def test_timeout_is_reported_and_context_survives():
    """A tile whose predecessor never publishes gives up after the bounded wait: the call reports
    MORLET_ERR_TIMEOUT and later launches on the same context still work."""
    import torch
    x = WL.white(4, 200000)
    plan = m.morlet_plan([len(x)], [3000.0], K=4, precision=m.MORLET_FP32_PLAIN, flags=m.MORLET_FLAG_NO_GRAPH)
    m.morlet_plan_set_spin_limit(plan, 2000)
    xt = torch.from_numpy(x).cuda()
    W = torch.empty(len(x), dtype=torch.complex64, device="cuda")
    m.morlet_debug_skip_tickets(plan, 1)   # work item 0 (the row's first tile) is never processed
    m.morlet_forward(plan, xt, W)
    assert m.morlet_last_device_error(plan) == m.MORLET_ERR_TIMEOUT
    m.morlet_forward(plan, xt, W)          # clean run afterwards
    assert m.morlet_last_device_error(plan) == 0
    ref = oracle_forward(x, 3000.0, 4)
    assert rel_err(W.cpu().numpy(), ref) < 1e-3


def test_prefix_sum_timeout_is_reported_and_context_survives():
    """The same for the warp-level look-back of the prefix-sum kernel (compensated FP32, a long
    window whose work items start from prefix sums)."""
    import torch
    x = WL.white(5, 300000)
    plan = m.morlet_plan([len(x)], [6000.0], K=4, precision=m.MORLET_FP32_COMP, flags=m.MORLET_FLAG_NO_GRAPH)
    st = m.morlet_plan_stats(plan)
    assert st["rows_start_state"] == 1 and st["prefix_items"] > 2 and st["start_state_window_sums"] == 0
    m.morlet_plan_set_spin_limit(plan, 2000)
    xt = torch.from_numpy(x).cuda()
    W = torch.empty(len(x), dtype=torch.complex64, device="cuda")
    m.morlet_debug_skip_tickets(plan, 1)   # the row's first chunk of prefix sums is never computed
    m.morlet_forward(plan, xt, W)
    assert m.morlet_last_device_error(plan) == m.MORLET_ERR_TIMEOUT
    m.morlet_forward(plan, xt, W)
    assert m.morlet_last_device_error(plan) == 0
    ref = oracle_forward(x, 6000.0, 4)
    assert rel_err(W.cpu().numpy(), ref) < 1e-5
