"""FP64 numpy oracle: fits, effective kernels and direct convolutions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Plain and slow on purpose: every step is the
paper's definition written out, with numpy's matmul / solve / convolve as the only primitives.

Notation follows the paper, with one rename: the paper's half window K is called L here and its
number of Fourier terms P (or P_D) is called K. beta = pi / L (Sec. II-A).
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------------------------
# Window, harmonics and phases
# ----------------------------------------------------------------------------------------------


def window_half(sigma: float, window_mult: float = 4.0) -> int:
    """Half window L = ceil(window_mult * sigma); the window is k in [-L, L] (Sec. II, eq. xG)."""
    return int(math.ceil(window_mult * sigma))


def harmonic_angle(p: int, k, L: int):
    """beta*p*k reduced exactly: pi * ((p*k) mod 2L) / L, so no large angle reaches cos/sin.

    beta = pi/L (Sec. II-A); the reduction is exact integer arithmetic because
    e^{i beta p 2L} = 1.
    """
    k = np.asarray(k, dtype=np.int64)
    r = np.mod(np.int64(p) * k, np.int64(2 * L))
    return np.pi * r.astype(np.float64) / float(L)


# ----------------------------------------------------------------------------------------------
# Target functions (Sec. II, Sec. III)
# ----------------------------------------------------------------------------------------------


def gaussian(k, sigma: float):
    """G[n] = sqrt(gamma/pi) exp(-gamma n^2), gamma = 1/(2 sigma^2) (Sec. II, first equation)."""
    g = 1.0 / (2.0 * sigma * sigma)
    k = np.asarray(k, dtype=np.float64)
    return math.sqrt(g / math.pi) * np.exp(-g * k * k)


def gaussian_d(k, sigma: float):
    """G_D[n] = (-2 gamma n) G[n] (Sec. II)."""
    g = 1.0 / (2.0 * sigma * sigma)
    k = np.asarray(k, dtype=np.float64)
    return (-2.0 * g * k) * gaussian(k, sigma)


def gaussian_dd(k, sigma: float):
    """G_DD[n] = (4 gamma^2 n^2 - 2 gamma) G[n] (Sec. II)."""
    g = 1.0 / (2.0 * sigma * sigma)
    k = np.asarray(k, dtype=np.float64)
    return (4.0 * g * g * k * k - 2.0 * g) * gaussian(k, sigma)


def morlet_constants(xi: float):
    """C_xi = (1 + e^{-xi^2} - 2 e^{-3 xi^2 / 4})^{-1/2}, kappa_xi = e^{-xi^2/2} (Sec. III)."""
    C = (1.0 + math.exp(-xi * xi) - 2.0 * math.exp(-0.75 * xi * xi)) ** -0.5
    kappa = math.exp(-0.5 * xi * xi)
    return C, kappa


def morlet(k, sigma: float, xi: float, norm: int = 0):
    """Discrete Morlet wavelet psi_{sigma,xi}[k] (Sec. III).

    norm = 0: the unnormalised form e^{-k^2/(2 sigma^2)} e^{i omega0 k}, omega0 = xi/sigma.
    norm = 1: C_xi pi^{-1/4} sigma^{-1/2} e^{-k^2/(2 sigma^2)} (e^{i xi k/sigma} - kappa_xi).
    The printed discrete formula is garbled (pi^{-1/4} sits in a denominator and the exponent
    uses t); this is the dilation of the continuous definition, the reading we take.
    """
    k = np.asarray(k, dtype=np.float64)
    env = np.exp(-k * k / (2.0 * sigma * sigma))
    w0 = xi / sigma
    if norm == 0:
        return env * np.exp(1j * w0 * k)
    C, kappa = morlet_constants(xi)
    return C * math.pi ** -0.25 / math.sqrt(sigma) * env * (np.exp(1j * w0 * k) - kappa)


# ----------------------------------------------------------------------------------------------
# Least-squares fits (eq. mmse; direct method of Sec. III-A)
# ----------------------------------------------------------------------------------------------


def _ls_fit(basis, target, L: int, ps, chunk: int = 1 << 20):
    """Minimise sum_{k=-L}^{L} |sum_p c_p basis(p,k) - target(k)|^2 (eq. mmse).

    Normal equations accumulated over chunks of k, solved with numpy.linalg.solve. Basis
    columns that vanish identically (sin with p = 0) are left out and get coefficient 0.
    Returns (coefficients, residual sum of squares).
    """
    ps = list(ps)
    keep = [i for i, p in enumerate(ps) if not (basis is np.sin and p == 0)]
    K = len(keep)
    G = np.zeros((K, K))
    b = np.zeros(K)
    yy = 0.0
    for k0 in range(-L, L + 1, chunk):
        k = np.arange(k0, min(k0 + chunk, L + 1), dtype=np.int64)
        A = np.stack([basis(harmonic_angle(ps[i], k, L)) for i in keep], axis=1)
        y = target(k)
        G += A.T @ A
        b += A.T @ y
        yy += float(y @ y)
    c = np.linalg.solve(G, b) if K else np.zeros(0)
    rss = yy - 2.0 * float(c @ b) + float(c @ G @ c)
    out = np.zeros(len(ps))
    out[keep] = c
    return out, max(rss, 0.0)


def candidate_starts(sigma: float, xi: float, K: int, L: int):
    """P_S candidates: [max(0, pc - K), pc] with pc = floor(omega0 / beta + 1/2).

    The paper picks the RMSE-optimal P_S (Fig. MSE2) without a rule; this range always holds
    the K harmonics centred on the carrier omega0 = xi / sigma.
    """
    pc = int(math.floor((xi / sigma) * L / math.pi + 0.5))
    return list(range(max(0, pc - K), pc + 1))


def fit_direct(sigma: float, xi: float, K: int, L: int | None = None, norm: int = 0,
               p_start: int | None = None):
    """Direct method (Sec. III-A): psi[k] ~ sum_{p=P_S}^{P_S+K-1} (m_p cos(beta p k) + i l_p sin(beta p k)).

    m_p fits Re psi (even) with cosines, l_p fits Im psi (odd) with sines, each by eq. mmse on
    k in [-L, L]. If p_start is None, P_S is the candidate with the smallest total residual
    (ties go to the smaller P_S). Returns dict(p0, m, l, L, rss).
    Pinned by: residual orthogonality, the orthogonal-grid closed form, Table I (soft) and the
    closed-form response tests in tests/test_oracle_pins.py.
    """
    L = window_half(sigma) if L is None else L
    starts = [p_start] if p_start is not None else candidate_starts(sigma, xi, K, L)
    best = None
    for p0 in starts:
        ps = range(p0, p0 + K)
        m, r1 = _ls_fit(np.cos, lambda k: morlet(k, sigma, xi, norm).real, L, ps)
        l, r2 = _ls_fit(np.sin, lambda k: morlet(k, sigma, xi, norm).imag, L, ps)
        r = r1 + r2
        if best is None or r < best["rss"]:
            best = dict(p0=p0, m=m, l=l, L=L, rss=r)
    return best


def fit_gauss(sigma: float, P: int, deriv: int, L: int | None = None):
    """Fourier-series fits of G, G_D, G_DD on [-L, L] (eq. aproGauss and the two after it).

    deriv 0: G ~ sum_{p=0}^{P} a_p cos(beta p k); deriv 1: G_D ~ sum_{p=1}^{P} b_p sin(beta p k);
    deriv 2: G_DD ~ sum_{p=0}^{P} d_p cos(beta p k). Returns dict(p0=0, coef, basis, L).
    """
    L = window_half(sigma) if L is None else L
    ps = range(0, P + 1)
    if deriv == 0:
        c, r = _ls_fit(np.cos, lambda k: gaussian(k, sigma), L, ps)
        return dict(p0=0, coef=c, basis="cos", L=L, rss=r)
    if deriv == 1:
        c, r = _ls_fit(np.sin, lambda k: gaussian_d(k, sigma), L, ps)
        return dict(p0=0, coef=c, basis="sin", L=L, rss=r)
    if deriv == 2:
        c, r = _ls_fit(np.cos, lambda k: gaussian_dd(k, sigma), L, ps)
        return dict(p0=0, coef=c, basis="cos", L=L, rss=r)
    raise ValueError("deriv must be 0, 1 or 2")


def fit_gauss_asft(sigma: float, P: int, deriv: int, n0: int, L: int | None = None):
    """Fits for Gaussian smoothing by the ASFT (eqs. GsASFT and gddAsft).

    The ASFT window weights x[n - k] by e^{-alpha k}, alpha = n0 / sigma^2. By the shift identity
    eq. siftGauss, e^{-alpha k} G[k] = e^{alpha^2/(4 gamma)} G[k + n0], so with
    C = e^{-alpha^2/(4 gamma)} and the derivative rule d/dk applied to k + n0:
        G[k + n0]    = C e^{-alpha k} G[k],
        G_D[k + n0]  = C e^{-alpha k} (G_D[k] - alpha G[k]),
        G_DD[k + n0] = C e^{-alpha k} (G_DD[k] - 2 alpha G_D[k] + alpha^2 G[k]).
    The printed eq. gddAsft carries these terms with misplaced factors and tildes; this is the
    reading taken. The bracket h is fitted on [-L, L] as in eq. mmse: its even part by
    cos(beta p k), its odd part by sin(beta p k), p = 0 .. P. Returns dict(L, n0, alpha, cos, sin).
    """
    L = window_half(sigma) if L is None else L
    alpha = asft_alpha(sigma, n0)
    ps = range(0, P + 1)
    if deriv == 0:
        even, odd = (lambda k: gaussian(k, sigma)), None
    elif deriv == 1:
        even, odd = (lambda k: -alpha * gaussian(k, sigma)), (lambda k: gaussian_d(k, sigma))
    elif deriv == 2:
        even = lambda k: gaussian_dd(k, sigma) + alpha * alpha * gaussian(k, sigma)
        odd = lambda k: -2.0 * alpha * gaussian_d(k, sigma)
    else:
        raise ValueError("deriv must be 0, 1 or 2")
    c, r1 = _ls_fit(np.cos, even, L, ps)
    if odd is None:
        sn, r2 = np.zeros(len(ps)), 0.0
    else:
        sn, r2 = _ls_fit(np.sin, odd, L, ps)
    return dict(L=L, n0=int(n0), alpha=alpha, sigma=float(sigma), cos=c, sin=sn, rss=r1 + r2)


def kernel_gauss_asft(gf):
    """Effective kernel of the ASFT Gaussian fit, on k' in [n0 - L, n0 + L]:
    C e^{-alpha (k' - n0)} h_hat[k' - n0], h_hat[k] = sum_p cos_p cos(beta p k) + sin_p sin(beta p k).
    Equal to G_X[k'] up to the fit residual. Returns (k', kernel)."""
    L, n0, alpha, sigma = gf["L"], gf["n0"], gf["alpha"], gf["sigma"]
    g = 1.0 / (2.0 * sigma * sigma)
    C = math.exp(-alpha * alpha / (4.0 * g))
    kk = np.arange(-L, L + 1, dtype=np.int64)
    h = np.zeros(kk.shape, np.float64)
    for p, (a, b) in enumerate(zip(gf["cos"], gf["sin"])):
        ang = harmonic_angle(p, kk, L)
        h += a * np.cos(ang) + b * np.sin(ang)
    return kk + n0, C * np.exp(-alpha * kk.astype(np.float64)) * h


def gauss_asft_direct(x, gf, n_idx=None):
    """Gaussian smoothing (or a derivative) by the ASFT fit: sum_{k'} kernel[k'] x[n - k']."""
    kp, ker = kernel_gauss_asft(gf)
    return conv_direct(x, ker, int(kp[0]), n_idx)


def fit_multiply(sigma: float, xi: float, K: int, L: int | None = None, norm: int = 0):
    """Multiplication method (Sec. III-B) for the unnormalised Morlet (norm = 0).

    The envelope e^{-k^2/(2 sigma^2)} is fitted on [-L, L] by sum_{p=0}^{K-1} a_p cos(beta p k)
    (eq. mmse); then psi[k] ~ sum_{p=-(K-1)}^{K-1} a'_p e^{i (omega0 + beta p) k} with a'_0 = a_0 and
    a'_{+-p} = a_p / 2 (the two-sided form of the cosine series). The kappa terms of the normalised
    Morlet are not part of the GPU build; with norm = 1 the oracle kernel includes them:
    C_xi pi^{-1/4} sigma^{-1/2} G_hat[k] (e^{i omega0 k} - kappa_xi), the kappa part being the
    harmonic series itself. Returns dict(L, sigma, xi, omega0, a, rss, norm).
    """
    L = window_half(sigma) if L is None else L
    a, r = _ls_fit(np.cos, lambda k: np.exp(-k.astype(np.float64) ** 2 / (2.0 * sigma * sigma)), L, range(K))
    return dict(L=L, sigma=float(sigma), xi=float(xi), omega0=float(xi) / sigma, a=a, rss=r, norm=norm)


def kernel_multiply(mf, k=None):
    """psi_mult[k] = sum_{p=-P}^{P} a'_p e^{i (omega0 + beta p) k}, P = K - 1, on k in [-L, L], summed
    term by term over the 2P + 1 non-harmonic frequencies omega0 + beta p."""
    L = mf["L"]
    k = np.arange(-L, L + 1, dtype=np.int64) if k is None else np.asarray(k, np.int64)
    a = mf["a"]
    P = len(a) - 1
    carrier = np.exp(1j * mf["omega0"] * k.astype(np.float64))
    out = np.zeros(k.shape, np.complex128)
    for p in range(-P, P + 1):
        ap = a[0] if p == 0 else 0.5 * a[abs(p)]
        out += ap * carrier * np.exp(1j * harmonic_angle(p, k, L))
    if mf.get("norm", 0):
        C, kappa = morlet_constants(mf["xi"])
        env_hat = sum(c * np.cos(harmonic_angle(p, k, L)) for p, c in enumerate(a))
        out = C * math.pi ** -0.25 / math.sqrt(mf["sigma"]) * (out - kappa * env_hat)
    return out


def morlet_multiply_direct(x, mf, n_idx=None):
    """Oracle for the multiplication method: sum_{k=-L}^{L} psi_mult[k] x[n-k]."""
    return conv_direct(x, kernel_multiply(mf), -mf["L"], n_idx)


# ----------------------------------------------------------------------------------------------
# Approximation error of the Morlet wavelet (Sec. IV, "Approximation error of the Morlet wavelet")
# ----------------------------------------------------------------------------------------------


def morlet_relative_rmse(kernel_hat, L: int, sigma: float, xi: float, norm: int = 1) -> float:
    """Relative RMSE of an approximated Morlet given on [-L, L] (zero outside) against the true
    psi_{sigma,xi}, both summed over n in [-5L, 5L] (the paper's definition)."""
    n = np.arange(-5 * L, 5 * L + 1)
    psi = morlet(n, sigma, xi, norm)
    hat = np.zeros(n.shape, np.complex128)
    hat[4 * L: 6 * L + 1] = kernel_hat
    return float(np.sqrt(np.sum(np.abs(hat - psi) ** 2) / np.sum(np.abs(psi) ** 2)))


def approx_error(method: str, sigma: float, xi: float, P: int, L: int, norm: int = 1):
    """Relative RMSE of one approximation at one window: method "direct" (P terms, least-residual
    P_S), "multiply" (2P + 1 non-harmonic terms from P + 1 envelope terms) or "truncated" (the
    true Morlet cut to [-L, L]). Returns (rmse, P_S or None)."""
    k = np.arange(-L, L + 1)
    if method == "direct":
        fit = fit_direct(sigma, xi, P, L, norm)
        return morlet_relative_rmse(kernel_direct(fit), L, sigma, xi, norm), fit["p0"]
    if method == "multiply":
        mf = fit_multiply(sigma, xi, P + 1, L, norm)
        return morlet_relative_rmse(kernel_multiply(mf), L, sigma, xi, norm), None
    if method == "truncated":
        return morlet_relative_rmse(morlet(k, sigma, xi, norm), L, sigma, xi, norm), None
    raise ValueError(method)


def best_window(method: str, sigma: float, xi: float, P: int, norm: int = 1,
                lo_mult: float = 2.0, hi_mult: float = 6.0, coarse: int = 8):
    """The window L in [lo_mult sigma, hi_mult sigma] with the smallest relative RMSE (the paper
    chooses the window that way): a scan with step `coarse`, refined by single steps around the best
    coarse point. The truncated Morlet keeps the paper's fixed interval [-3 sigma, 3 sigma].
    Returns dict(L, rmse, p0)."""
    if method == "truncated":
        L = int(round(3.0 * sigma))
        r, _ = approx_error(method, sigma, xi, P, L, norm)
        return dict(L=L, rmse=r, p0=None)
    lo, hi = int(math.ceil(lo_mult * sigma)), int(math.floor(hi_mult * sigma))
    best = None
    def visit(L):
        nonlocal best
        r, p0 = approx_error(method, sigma, xi, P, L, norm)
        if best is None or r < best["rmse"]:
            best = dict(L=L, rmse=r, p0=p0)
    for L in range(lo, hi + 1, coarse):
        visit(L)
    c = best["L"]
    for L in range(max(lo, c - coarse + 1), min(hi, c + coarse - 1) + 1):
        if L != c:
            visit(L)
    return best


# ----------------------------------------------------------------------------------------------
# Effective kernels: what each method computes exactly (up to rounding)
# ----------------------------------------------------------------------------------------------


def kernel_direct(fit, k=None):
    """psi_hat[k] = sum_p (m_p cos(beta p k) + i l_p sin(beta p k)) on k in [-L, L] (Sec. III-A).

    The SFT method returns exactly sum_k psi_hat[k] x[n-k]; that sum is the oracle's definition.
    """
    L = fit["L"]
    k = np.arange(-L, L + 1, dtype=np.int64) if k is None else np.asarray(k, np.int64)
    out = np.zeros(k.shape, np.complex128)
    for j, (m, l) in enumerate(zip(fit["m"], fit["l"])):
        a = harmonic_angle(fit["p0"] + j, k, L)
        out += m * np.cos(a) + 1j * l * np.sin(a)
    return out


def kernel_gauss(gfit, k=None):
    """G_hat_X[k] = sum_p coef_p cos(beta p k) (or sin) on [-L, L] (eq. aproGauss)."""
    L = gfit["L"]
    k = np.arange(-L, L + 1, dtype=np.int64) if k is None else np.asarray(k, np.int64)
    fn = np.cos if gfit["basis"] == "cos" else np.sin
    out = np.zeros(k.shape, np.float64)
    for j, c in enumerate(gfit["coef"]):
        out += c * fn(harmonic_angle(gfit["p0"] + j, k, L))
    return out


def asft_alpha(sigma: float, n0: int) -> float:
    """alpha = 2 gamma n0 = n0 / sigma^2, so that n0 = alpha / (2 gamma) is the integer shift (Sec. II-E)."""
    return float(n0) / (sigma * sigma)


def default_n0(sigma: float) -> int:
    """ASFT shift when none is given: max(1, round(sigma / 8)).

    The paper uses n0 = 10 at L = 256 for Table I and gives no rule for the Morlet transform.
    This choice keeps the decay memory 1/alpha = 8 sigma and the edge gain e^{alpha L} = e^{1/2}
    independent of sigma.
    """
    return max(1, int(math.floor(sigma / 8.0 + 0.5)))


def kernel_asft(fit, sigma: float, xi: float, n0: int):
    """Effective kernel of the ASFT direct method, on k' in [n0 - L, n0 + L].

    The ASFT components weight x[n-k] by e^{-alpha k} (the decaying reading of eqs. acp/asp: the
    recursion eq. iir1A damps older samples). With the shift identity eq. siftGauss,
    e^{-alpha k} G[k] = e^{alpha^2/(4 gamma)} G[k + n0], the Morlet output is
        x_M[n] = E * sum_p (m_p c~_p + i l_p s~_p)[n - n0],  E = e^{-alpha^2/(4 gamma)} e^{i omega0 n0},
    i.e. sum_{k'} psi~[k'] x[n - k'] with psi~[k'] = E e^{-alpha (k'-n0)} psi_hat[k' - n0].
    The carrier factor e^{i omega0 n0} is not printed in the paper; without it the output is off
    by a constant phase. Returns (k', psi~[k']).
    """
    L = fit["L"]
    alpha = asft_alpha(sigma, n0)
    g = 1.0 / (2.0 * sigma * sigma)
    E = math.exp(-alpha * alpha / (4.0 * g)) * np.exp(1j * (xi / sigma) * n0)
    kk = np.arange(-L, L + 1, dtype=np.int64)
    kp = kk + n0
    return kp, E * np.exp(-alpha * kk.astype(np.float64)) * kernel_direct(fit, kk)


# ----------------------------------------------------------------------------------------------
# Direct convolutions (the definitions)
# ----------------------------------------------------------------------------------------------


def conv_direct(x, kern, kmin: int, n_idx=None):
    """W[n] = sum_k kern(k) x[n-k] over k in [kmin, kmin + len(kern)), x zero outside [0, N).

    Full output via numpy.convolve (a direct O(N * len) sum); or only at the sample indices
    n_idx, each by one dot product. Complex kernels are split into real and imaginary parts.
    """
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    kern = np.asarray(kern)
    M = kern.shape[0]
    if n_idx is None:
        def cv(h):
            full = np.convolve(x, h)               # full[i] = sum_j x[j] h[i - j]
            # W[n] = sum_k h[k - kmin] x[n - k] = full[n - kmin]
            out = np.zeros(N)
            lo = -kmin
            src = np.arange(N) + lo
            ok = (src >= 0) & (src < full.shape[0])
            out[ok] = full[src[ok]]
            return out
        if np.iscomplexobj(kern):
            return cv(kern.real) + 1j * cv(kern.imag)
        return cv(kern)
    n_idx = np.asarray(n_idx, dtype=np.int64)
    out = np.zeros(n_idx.shape, dtype=np.complex128 if np.iscomplexobj(kern) else np.float64)
    for i, n in enumerate(n_idx):
        k_lo = max(kmin, n - N + 1)
        k_hi = min(kmin + M - 1, n)
        if k_hi < k_lo:
            continue
        ks = np.arange(k_lo, k_hi + 1)
        out[i] = np.dot(kern[ks - kmin], x[n - ks])
    return out


def morlet_sft_direct(x, fit, n_idx=None):
    """Oracle O-direct: the SFT direct-method Morlet transform as sum_{k=-L}^{L} psi_hat[k] x[n-k]."""
    return conv_direct(x, kernel_direct(fit), -fit["L"], n_idx)


def morlet_asft_direct(x, fit, sigma: float, xi: float, n0: int, n_idx=None):
    """Oracle for the ASFT direct method: sum_{k'} psi~[k'] x[n-k'] (see kernel_asft)."""
    kp, ker = kernel_asft(fit, sigma, xi, n0)
    return conv_direct(x, ker, int(kp[0]), n_idx)


def morlet_true_direct(x, sigma: float, xi: float, norm: int = 0, half_mult: float = 8.0,
                       n_idx=None):
    """Direct convolution with the true Morlet wavelet truncated at +-ceil(8 sigma)."""
    H = int(math.ceil(half_mult * sigma))
    k = np.arange(-H, H + 1)
    return conv_direct(x, morlet(k, sigma, xi, norm), -H, n_idx)


def gauss_sft_direct(x, gfit, n_idx=None):
    """Gaussian smoothing (or a derivative) by the fitted kernel: sum_k G_hat_X[k] x[n-k] (eq. GsSFT)."""
    return conv_direct(x, kernel_gauss(gfit), -gfit["L"], n_idx)


def edge_extended(x, E: int):
    """x extended by E copies of its first and last values (the "values on the edges" boundary of
    Sec. II): a transform of this array at positions [E, E + N) is the edge-extended transform of x,
    provided E covers the window's reach."""
    return np.pad(np.asarray(x), (E, E), mode="edge")


def gauss_filter_2d_direct(img, sigma: float, P: int, deriv_y: int, deriv_x: int):
    """Separable 2-D Gaussian filtering (Sec. IV, 2-D signals as independent rows and columns): the
    fitted 1-D kernel of eq. GsSFT (or its derivative form) convolved along every row (deriv_x),
    then along every column (deriv_y); zero extension outside the image."""
    img = np.asarray(img, dtype=np.float64)
    gx, gy = fit_gauss(sigma, P, deriv_x), fit_gauss(sigma, P, deriv_y)
    rows = np.stack([gauss_sft_direct(r, gx) for r in img])
    return np.stack([gauss_sft_direct(c, gy) for c in rows.T]).T


def adjoint_direct(g, fit, n_idx=None):
    """Transpose of x -> W = sum_k psi_hat[k] x[n-k] for real x and a real loss.

    With g[n] = dLoss/dRe W[n] + i dLoss/dIm W[n], the gradient is
        dx[t] = sum_n Re(conj(g[n]) dW[n]/dx[t]) = sum_{k=-L}^{L} Re(conj(g[t+k]) psi_hat[k]),
    g zero outside [0, N). Pinned by the inner-product identity
    sum_n Re(conj(g[n]) W[n]) = sum_t x[t] dx[t] and by central finite differences.
    """
    g = np.asarray(g, dtype=np.complex128)
    N = g.shape[0]
    L = fit["L"]
    ker = kernel_direct(fit)                      # ker[k + L] = psi_hat[k]
    if n_idx is None:
        rev = ker[::-1]                           # rev[i] = psi_hat[L - i]
        gc = np.conj(g)
        # S[t] = sum_k conj(g[t+k]) psi_hat[k] = sum_i conj(g)[t + L - i] rev[i] = (conj(g) * rev)[t + L]
        full = np.convolve(gc.real, rev.real) - np.convolve(gc.imag, rev.imag) \
            + 1j * (np.convolve(gc.real, rev.imag) + np.convolve(gc.imag, rev.real))
        return full[L:L + N].real
    out = np.zeros(len(n_idx))
    for i, t in enumerate(np.asarray(n_idx, np.int64)):
        ks = np.arange(max(-L, -t), min(L, N - 1 - t) + 1)
        out[i] = float(np.sum((np.conj(g[t + ks]) * ker[ks + L]).real))
    return out


# ----------------------------------------------------------------------------------------------
# Errors, Table I and Algorithm 1
# ----------------------------------------------------------------------------------------------


def relative_rmse(approx, exact):
    """sqrt(sum |approx - exact|^2 / sum |exact|^2) (eq. mmseGEx)."""
    a = np.asarray(approx)
    e = np.asarray(exact)
    return math.sqrt(float(np.sum(np.abs(a - e) ** 2)) / float(np.sum(np.abs(e) ** 2)))


def table1_sft_rmse(P: int, deriv: int, L: int = 256, sigma: float | None = None,
                    beta: float | None = None):
    """Relative RMSE of the SFT Gaussian fit as in Table I: L = 256, error summed over [-3L, 3L]
    with the approximation set to 0 outside [-L, L] (eq. mmseGEx). sigma and beta are not printed;
    sigma defaults to L/3 ("K is close to 3 sigma") and beta to pi/L when not given."""
    sigma = L / 3.0 if sigma is None else sigma
    beta = math.pi / L if beta is None else beta
    k = np.arange(-L, L + 1, dtype=np.float64)
    ps = list(range(0, P + 1)) if deriv != 1 else list(range(1, P + 1))
    fn = np.sin if deriv == 1 else np.cos
    tgt = [gaussian, gaussian_d, gaussian_dd][deriv]
    A = np.stack([fn(beta * p * k) for p in ps], axis=1)
    c = np.linalg.solve(A.T @ A, A.T @ tgt(k, sigma))
    kk = np.arange(-3 * L, 3 * L + 1, dtype=np.float64)
    approx = np.where(np.abs(kk) <= L, np.stack([fn(beta * p * kk) for p in ps], axis=1) @ c, 0.0)
    return relative_rmse(approx, tgt(kk, sigma))


def table1_best_beta(P: int, L: int = 256, sigma: float | None = None, lo=0.5, hi=1.6, iters=60):
    """Golden-section search of beta = f * pi / L minimising the Table I e(G) (the paper optimises beta per P)."""
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    f = lambda s: table1_sft_rmse(P, 0, L, sigma, s * math.pi / L)
    a, b = lo, hi
    c, d = b - gr * (b - a), a + gr * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - gr * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + gr * (b - a)
            fd = f(d)
    s = 0.5 * (a + b)
    return s * math.pi / L


def sliding_sum_doubling(f, length: int):
    """Algorithm 1 (basic doubling sliding sum) restated on the CPU: h[n] = sum_{k=0}^{length-1} f[n+k].

    g holds sums of 2^r consecutive samples; whenever bit r of `length` is set, h takes g plus
    the part already accumulated 2^r further on. Valid for n = 0 .. N - length.
    """
    f = np.asarray(f)
    N = f.shape[0]
    R = max(1, int(length).bit_length())
    g = f.copy()
    h = np.zeros_like(f)
    for r in range(R):
        s = 1 << r
        # samples past the end count as zero, so the last valid window n = N - length is complete
        if (length >> r) & 1:
            hn = g.copy()
            hn[:N - s] += h[s:]
            h = hn
        gn = g.copy()
        gn[:N - s] += g[s:]
        g = gn
    return h[:N - length + 1]
