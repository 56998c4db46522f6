"""CPU checks (numpy, FP64) of the algebraic rewritings the warp-scan kernels run, against the plain
recursions they replace. The kernels' outputs are checked against the oracle on the GPU; these
tests pin the identities themselves, so that a slip in a derivation (a sign, a factor r, an index
of s) fails here with a readable message.

- Pass 1 of the SFT (Sec. II-C): G <- rho G + d from zero over 16 samples, rho = e^{-i theta}, as
  Reinsch's second-order recurrence e_i = e_{i-1} + d_i - lam s_{i-1}, s_i = s_{i-1} + e_i,
  G = (e_15 + (lam / 2) s_14) + i Im(rho) s_14, lam = 4 sin^2(theta / 2).
- Pass 1 of the ASFT (Sec. II-D): the same for a damped rotation rho = r e^{-i theta}:
  e_i = r e_{i-1} + d_i - r lam s_{i-1}, s_i = r s_{i-1} + e_i, U = (e_15 + (r lam / 2) s_14)
  + i Im(rho) s_14.
- The ASFT's U form: with kappa = rho^{2L} real, V <- rho (V - kappa x[t - 2L - 1]) + x[t] (the
  window of the last 2L + 1 samples) and U = V - kappa x[t - 2L] obey
  U <- rho U + (x[t] - kappa x[t - 2L]).
- The SFT warp scan in the frame of the tile start: with lane aggregates B_l, B'_l =
  rho^{-16 (l + 1)} B_l, the state before lane l is rho^{16 l} (C + sum_{l' < l} B'_{l'}).
- Start states from tile sums: the window sum ending at t_a - 1 is sum_k rho^{512 (kb - 1 - k)} G_k
  over the tiles inside the window, plus the masked part of the tile holding its first sample.
- The three-shear rotation x += t y, y -= s x, x += t y with t = tan(theta / 2), s = sin(theta)
  multiplies x + i y by e^{-i theta}.
"""
import numpy as np


def complex_pass(rho, d):
    g = 0j
    for v in d:
        g = rho * g + v
    return g


def reinsch_pass(theta, d):
    lam = 4.0 * np.sin(theta / 2) ** 2
    e = s = 0.0
    s_prev = 0.0
    for i, v in enumerate(d):
        e_new = e + v - lam * s
        s_prev = s
        s = s + e_new
        e = e_new
    s14 = s_prev
    return (e + 0.5 * lam * s14) + 1j * (-np.sin(theta)) * s14


def damped_reinsch_pass(r, theta, d):
    lam = 4.0 * np.sin(theta / 2) ** 2
    e = s = 0.0
    s_prev = 0.0
    for v in d:
        e_new = r * e + v - r * lam * s
        s_prev = s
        s = r * s + e_new
        e = e_new
    s14 = s_prev
    rho = r * np.exp(-1j * theta)
    return (e + 0.5 * r * lam * s14) + 1j * rho.imag * s14


def test_reinsch_pass_equals_the_rotation():
    rng = np.random.default_rng(5)
    for _ in range(200):
        theta = rng.choice([rng.uniform(1e-5, 1e-2), rng.uniform(0.01, np.pi)])
        d = rng.standard_normal(16)
        want = complex_pass(np.exp(-1j * theta), d)
        got = reinsch_pass(theta, d)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (theta, got, want)


def test_damped_reinsch_pass_equals_the_damped_rotation():
    rng = np.random.default_rng(6)
    for _ in range(200):
        theta = rng.choice([rng.uniform(1e-5, 1e-2), rng.uniform(0.01, np.pi)])
        r = np.exp(-rng.uniform(1e-6, 0.2))
        d = rng.standard_normal(16)
        want = complex_pass(r * np.exp(-1j * theta), d)
        got = damped_reinsch_pass(r, theta, d)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (r, theta, got, want)
    # r = 1 reduces to the undamped form
    d = rng.standard_normal(16)
    assert abs(damped_reinsch_pass(1.0, 0.3, d) - reinsch_pass(0.3, d)) < 1e-13


def test_asft_u_form_tracks_the_v_recursion():
    rng = np.random.default_rng(7)
    for L in (1, 5, 32):
        p, alpha = 3, 0.01
        beta = np.pi / L
        rho = np.exp(-alpha) * np.exp(-1j * beta * p)
        kappa = rho ** (2 * L)
        assert abs(kappa.imag) < 1e-12  # beta p 2L is a whole number of turns
        kappa = kappa.real
        x = rng.standard_normal(400)
        xa = lambda t: x[t] if 0 <= t < len(x) else 0.0
        V = 0j
        U = 0j
        for t in range(len(x)):
            V = rho * (V - kappa * xa(t - 2 * L - 1)) + xa(t)
            U = rho * U + (xa(t) - kappa * xa(t - 2 * L))
            assert abs(U - (V - kappa * xa(t - 2 * L))) < 1e-10, (L, t)
        # and V is the damped window sum of the last 2L + 1 samples
        t = len(x) - 1
        win = sum(rho ** (t - u) * xa(u) for u in range(t - 2 * L, t + 1))
        assert abs(V - win) < 1e-10


def test_frame_of_tile_scan_gives_each_lanes_start_state():
    rng = np.random.default_rng(8)
    for theta in (1e-4, 0.37, 2.9):
        rho = np.exp(-1j * theta)
        C = complex(rng.standard_normal(), rng.standard_normal())
        d = rng.standard_normal(512)
        B = np.array([complex_pass(rho, d[16 * l:16 * l + 16]) for l in range(32)])
        Bp = rho ** (-16.0 * (np.arange(32) + 1)) * B
        excl = np.concatenate([[0j], np.cumsum(Bp)[:-1]])
        S = rho ** (16.0 * np.arange(32)) * (C + excl)
        g = C
        for l in range(32):
            assert abs(S[l] - g) < 1e-10 * max(1.0, abs(g)), (theta, l)
            for v in d[16 * l:16 * l + 16]:
                g = rho * g + v
        assert abs(rho ** 512 * (C + Bp.sum()) - g) < 1e-9 * max(1.0, abs(g))


def test_start_state_from_tile_sums_is_the_window_sum():
    rng = np.random.default_rng(9)
    T = 512
    for _ in range(20):
        L = int(rng.integers(1, 2000))
        theta = np.pi * int(rng.integers(1, 6)) / L
        rho = np.exp(-1j * theta)
        t_grid = -512 + int(rng.integers(0, 8))
        kb = int(rng.integers(1, 12))
        n = T * (kb + 2)
        x = rng.standard_normal(n)
        xa = lambda u: x[u] if 0 <= u < n else 0.0
        t_a = t_grid + T * kb
        u0 = t_a - 2 * L
        want = sum(rho ** (t_a - 1 - u) * xa(u) for u in range(max(u0, t_grid), t_a))
        # tile sums G_k = sum_{u in tile k} rho^{e_k - u} x[u], e_k the tile's last position
        def tile_sum(k, lo):
            a0 = t_grid + T * k
            return sum(rho ** (a0 + T - 1 - u) * xa(u) for u in range(max(a0, lo), a0 + T))
        k0 = (u0 - t_grid) // T if u0 > t_grid else 0
        got = 0j
        for k in range(k0, kb):
            got += rho ** (T * (kb - 1 - k)) * tile_sum(k, u0 if k == k0 else t_grid)
        assert abs(got - want) < 1e-9 * max(1.0, abs(want)), (L, kb, t_grid)


def test_three_shears_rotate_by_minus_theta():
    rng = np.random.default_rng(10)
    for theta in (1e-6, 0.01, 1.0, 3.0):
        t, s = np.tan(theta / 2), np.sin(theta)
        x0, y0 = rng.standard_normal(2)
        x, y = x0, y0
        x = x + t * y
        y = y - s * x
        x = x + t * y
        want = complex(x0, y0) * np.exp(-1j * theta)
        assert abs(complex(x, y) - want) < 1e-12, theta
