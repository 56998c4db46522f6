// Plan-time GPU work in FP64: the least-squares fit of the Fourier coefficients (eq. mmse, direct
// method of Sec. III-A, eq. aproGauss for Gaussian smoothing) and the per-scale tables the scan
// kernels read (steps, rotation powers, combine weights).
#include <math.h>

#include "common.cuh"
#include "plan_internal.h"

namespace msft {

// sum_{k=-L}^{L} cos(pi m k / L): 2L+1 when m = 0 mod 2L, otherwise (-1)^m
// (the 2L samples k = -L .. L-1 cover whole periods and sum to zero; k = L adds cos(pi m)).
__device__ double cos_sum(long long m, long long L) {
  long long mm = m % (2 * L);
  if (mm < 0) mm += 2 * L;
  if (mm == 0) return (double)(2 * L + 1);
  return (m & 1) ? -1.0 : 1.0;
}

// e^{i pi r / L} for the exact integer r = (p n) mod 2L
__device__ double2 harmonic(long long p, long long n, long long L) {
  long long r = (p % (2 * L)) * (n % (2 * L)) % (2 * L);
  if (r < 0) r += 2 * L;
  double s, c;
  sincospi((double)r / (double)L, &s, &c);
  return make_double2(c, s);
}

// Targets on k >= 0 (both are even after multiplying by the matching basis): tc pairs with cos,
// ts pairs with sin.
__device__ void fit_target(const FitJob& J, long long k, double* tc, double* ts) {
  const double kk = (double)k;
  if (J.method == 0) {  // Morlet (Sec. III)
    const double env = exp(-kk * kk / (2.0 * J.sigma * J.sigma));
    double s, c;
    sincos(J.omega0 * kk, &s, &c);
    *tc = J.amp * env * (c - J.kappa_xi);
    *ts = J.amp * env * s;
  } else if (J.method == 2) {  // multiplication method (Sec. III-B): the Morlet envelope alone
    *tc = J.amp * exp(-kk * kk / (2.0 * J.sigma * J.sigma));
    *ts = 0.0;
  } else {  // Gaussian and its derivatives (Sec. II)
    const double g = 1.0 / (2.0 * J.sigma * J.sigma);
    const double G = sqrt(g / M_PI) * exp(-g * kk * kk);
    const double GD = -2.0 * g * kk * G, GDD = (4.0 * g * g * kk * kk - 2.0 * g) * G;
    // ASFT (Sec. II-E): the damped window weights x[n - k] by e^{-alpha k}, and the shift identity
    // e^{-alpha k} G[k] = e^{alpha^2/(4 gamma)} G[k + n0] (n0 = alpha / (2 gamma)) turns the
    // derivatives into fixed mixtures: with C = e^{-alpha^2/(4 gamma)},
    //   G_D[k + n0]  = C e^{-alpha k} (G_D - alpha G)[k],
    //   G_DD[k + n0] = C e^{-alpha k} (G_DD - 2 alpha G_D + alpha^2 G)[k].
    // The fitted target is that mixture: its even part goes to the cos terms, its odd part to the
    // sin terms (alpha = 0 gives the SFT targets).
    const double a = J.alpha;
    if (J.deriv == 0) {
      *tc = G;
      *ts = 0.0;
    } else if (J.deriv == 1) {
      *tc = -a * G;
      *ts = GD;
    } else {
      *tc = GDD + a * a * G;
      *ts = -2.0 * a * GD;
    }
  }
}

// Stage 1: partial sums over a contiguous range of k in [0, L] for one scale per blockIdx.y.
// partial[(s * nblk + b) * FIT_STRIDE + ...] = {b_cos[h] (h < nh), b_sin[h], yy}.
__global__ void fit_partial(const FitJob* jobs, double* partial, int nblk) {
  const FitJob J = jobs[blockIdx.y];
  const long long L = J.L;
  const long long span = (L + 1 + nblk - 1) / nblk;
  const long long k0 = (long long)blockIdx.x * span;
  const long long k1 = min(L + 1, k0 + span);
  double bc[2 * KMAX], bs[2 * KMAX], yy = 0.0;
#pragma unroll
  for (int h = 0; h < 2 * KMAX; ++h) bc[h] = bs[h] = 0.0;
  for (long long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double w = (k == 0) ? 1.0 : 2.0;  // k and -k together
    double tc, ts;
    fit_target(J, k, &tc, &ts);
    yy += w * (tc * tc + ts * ts);
#pragma unroll
    for (int h = 0; h < 2 * KMAX; ++h) {
      if (h < J.nh) {
        const double2 e = harmonic(J.ph_lo + h, k, L);
        bc[h] += w * tc * e.x;
        bs[h] += w * ts * e.y;
      }
    }
  }
  // block reduction in a fixed order
  __shared__ double red[256];
  double* out = partial + ((size_t)blockIdx.y * nblk + blockIdx.x) * FIT_STRIDE;
  for (int q = 0; q < 2 * (2 * KMAX) + 1; ++q) {
    double v = (q < 2 * KMAX) ? bc[q] : (q < 4 * KMAX ? bs[q - 2 * KMAX] : yy);
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = red[0];
    __syncthreads();
  }
}

// Solve the K x K normal equations with the closed-form Gram matrix by Cholesky; returns the
// residual sum of squares yy - c.b, or -1 if the system is not positive definite.
__device__ double ls_solve(const long long* ps, int K, long long L, bool sine, const double* b, double yy,
                           double* c) {
  double A[KMAX][KMAX], y[KMAX];
  int idx[KMAX], n = 0;
  for (int i = 0; i < K; ++i) {
    c[i] = 0.0;
    if (sine && (ps[i] % L) == 0) continue;  // sin(pi p k / L) vanishes on integer k
    idx[n++] = i;
  }
  for (int a = 0; a < n; ++a)
    for (int q = 0; q < n; ++q) {
      const long long p = ps[idx[a]], r = ps[idx[q]];
      A[a][q] = sine ? 0.5 * (cos_sum(p - r, L) - cos_sum(p + r, L)) : 0.5 * (cos_sum(p - r, L) + cos_sum(p + r, L));
    }
  // Cholesky A = G G^T in place (lower)
  for (int j = 0; j < n; ++j) {
    double d = A[j][j];
    for (int q = 0; q < j; ++q) d -= A[j][q] * A[j][q];
    if (!(d > 0.0)) return -1.0;
    d = sqrt(d);
    A[j][j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = A[i][j];
      for (int q = 0; q < j; ++q) v -= A[i][q] * A[j][q];
      A[i][j] = v / d;
    }
  }
  for (int i = 0; i < n; ++i) {  // forward
    double v = b[idx[i]];
    for (int q = 0; q < i; ++q) v -= A[i][q] * y[q];
    y[i] = v / A[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {  // backward
    double v = y[i];
    for (int q = i + 1; q < n; ++q) v -= A[q][i] * c[idx[q]];
    c[idx[i]] = v / A[i][i];
  }
  double cb = 0.0;
  for (int i = 0; i < K; ++i) cb += c[i] * b[i];
  return yy - cb;
}

// Stage 2: one thread per scale sums the partials in block order, fits every candidate start
// (and every K when J.K == 0), keeps the least residual (ties -> smaller start), and writes the
// scale's fit into tab.
__global__ void fit_solve(const FitJob* jobs, const double* partial, int nblk, int n_scales, ScaleTab* tabs) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_scales) return;
  const FitJob J = jobs[s];
  double bc[2 * KMAX], bs[2 * KMAX], yy = 0.0;
  for (int h = 0; h < 2 * KMAX; ++h) bc[h] = bs[h] = 0.0;
  for (int b = 0; b < nblk; ++b) {
    const double* in = partial + ((size_t)s * nblk + b) * FIT_STRIDE;
    for (int h = 0; h < 2 * KMAX; ++h) {
      bc[h] += in[h];
      bs[h] += in[2 * KMAX + h];
    }
    yy += in[4 * KMAX];
  }
  ScaleTab& tb = tabs[s];
  int kbest = 0;
  long long p0best = 0;
  double rbest = -1.0, mbest[KMAX], lbest[KMAX];
  const int k_lo = J.K > 0 ? J.K : 1, k_hi = J.K > 0 ? J.K : KMAX;
  for (int K = k_lo; K <= k_hi; ++K) {
    long long s_lo, s_hi;
    if (J.method == 0) {
      s_lo = J.pc - K > 0 ? J.pc - K : 0;
      s_hi = J.pc;
    } else {
      s_lo = s_hi = 0;
    }
    double rk = -1.0, mk[KMAX], lk[KMAX];
    long long pk = 0;
    for (long long st = s_lo; st <= s_hi; ++st) {
      long long ps[KMAX];
      double bcs[KMAX], bss[KMAX], m[KMAX], l[KMAX];
      for (int j = 0; j < K; ++j) {
        ps[j] = st + j;
        bcs[j] = bc[st + j - J.ph_lo];
        bss[j] = bs[st + j - J.ph_lo];
      }
      double r;
      if (J.method == 0) {
        const double r1 = ls_solve(ps, K, J.L, false, bcs, 0.0, m);
        const double r2 = ls_solve(ps, K, J.L, true, bss, 0.0, l);
        r = yy + r1 + r2;  // yy - c.b over both parts
      } else if (J.alpha > 0.0 && J.deriv > 0) {  // ASFT derivative: both parts
        const double r1 = ls_solve(ps, K, J.L, false, bcs, 0.0, m);
        const double r2 = ls_solve(ps, K, J.L, true, bss, 0.0, l);
        r = yy + r1 + r2;
      } else if (J.deriv == 1) {
        r = yy + ls_solve(ps, K, J.L, true, bss, 0.0, l);
        for (int j = 0; j < K; ++j) m[j] = 0.0;
      } else {
        r = yy + ls_solve(ps, K, J.L, false, bcs, 0.0, m);
        for (int j = 0; j < K; ++j) l[j] = 0.0;
      }
      if (rk < 0.0 || r < rk) {
        rk = r;
        pk = st;
        for (int j = 0; j < K; ++j) {
          mk[j] = m[j];
          lk[j] = l[j];
        }
      }
    }
    kbest = K;
    p0best = pk;
    rbest = rk;
    for (int j = 0; j < K; ++j) {
      mbest[j] = mk[j];
      lbest[j] = lk[j];
    }
    // automatic K: stop at the first K whose relative RMSE meets the tolerance
    if (J.K == 0 && sqrt(fmax(rk, 0.0) / yy) <= J.fit_tol) break;
  }
  tb.p0 = (int32_t)p0best;
  tb.K = kbest;
  tb.rss = rbest;
  tb.yy = yy;
  for (int j = 0; j < KMAX; ++j) {
    tb.m[j] = j < kbest ? mbest[j] : 0.0;
    tb.l[j] = j < kbest ? lbest[j] : 0.0;
  }
}

// Per-scale tables for a kernel with `items` samples per thread. Rotating form:
// rho = e^{-alpha} e^{-i beta p}; kernel-integral form: rho = e^{+i beta p}. Every power rho^n is
// formed directly from the exact integer (p n) mod 2L and e^{-alpha n} (no repeated products).
__global__ void build_tables(ScaleTab* tabs, const FitJob* jobs, int n_scales, int K_kernel, int items, int form) {
  const int s = blockIdx.x;
  if (s >= n_scales) return;
  ScaleTab& tb = tabs[s];
  const FitJob J = jobs[s];
  const long long L = J.L;
  const double alpha = J.alpha;
  const bool rot = (form == 2);
  // multiplication method: term j < 2P + 1 has the non-harmonic frequency omega_j = omega0 +
  // beta (j - P), P = (Gaussian terms) - 1, and rho_j = e^{i omega_j}; its powers are e^{i omega0 n}
  // (FP64 angle) times the exact harmonic e^{i beta (j - P) n}. The normalised Morlet (kappa_xi != 0)
  // adds the terms j = 2P + 1 + q, q = 0..P, of the kappa part -kappa_xi sum_q m_q cos(beta q k): the
  // harmonics rho = e^{i beta q} with exact powers.
  const bool mult = (J.method == 2);
  const long long Pm = mult ? (long long)tb.K - 1 : 0;
  const long long n_morlet = 2 * Pm + 1;
  auto power = [&](long long p, long long n) -> double2 {
    if (mult) {
      const long long j = p - tb.p0;
      if (j >= n_morlet) return harmonic(j - n_morlet, n, L);
      double sn, cs;
      sincos(fmod(J.omega0 * (double)n, 2.0 * M_PI), &sn, &cs);
      const double2 h = harmonic(j - Pm, n, L);
      return make_double2(cs * h.x - sn * h.y, cs * h.y + sn * h.x);
    }
    const double2 e = harmonic(p, n, L);
    if (!rot) return e;
    const double a = exp(-alpha * (double)n);
    return make_double2(a * e.x, -a * e.y);
  };
  const long long T = (long long)THREADS * items;
  for (int idx = threadIdx.x; idx < K_kernel * (1 + 5 + 1 + 8 + 32 + 33); idx += blockDim.x) {
    const int j = idx % K_kernel;
    const int q = idx / K_kernel;
    const long long p = (long long)tb.p0 + j;
    if (q == 0) tb.rho[j] = power(p, 1);
    else if (q < 6) tb.pw_thr[q - 1][j] = power(p, (long long)items << (q - 1));
    else if (q == 6) tb.pw_warp[j] = power(p, (long long)items * 32);
    else if (q < 15) tb.pw_wofs[q - 7][j] = power(p, (long long)items * 32 * (q - 7));
    else if (q < 47) tb.pw_lane[q - 15][j] = power(p, (long long)items * (q - 15));
    else tb.pw_tile[q - 47][j] = power(p, T * (q - 47));
  }
  __syncthreads();
  auto dfc4 = [](double2 v) {
    const float rh = (float)v.x, ih = (float)v.y;
    return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
  };
  for (int idx = threadIdx.x; idx < K_kernel * 33; idx += blockDim.x)
    tb.c_pw_tile[idx / K_kernel][idx % K_kernel] = dfc4(tb.pw_tile[idx / K_kernel][idx % K_kernel]);
  for (int idx = threadIdx.x; idx < K_kernel * 48; idx += blockDim.x) {  // e^{+i beta p n} = rho^{-n}
    const int j = idx % K_kernel, q = idx / K_kernel;
    const long long p = (long long)tb.p0 + j;
    if (q < 32) tb.c_neg16[q][j] = dfc4(harmonic(p, 16LL * q, L));
    else tb.c_neg1[q - 32][j] = dfc4(harmonic(p, (long long)(q - 32), L));
  }
  for (int j = threadIdx.x; j < KMAX; j += blockDim.x) {
    double sh, ch;
    sincospi((double)(tb.p0 + j) / (double)(2 * L), &sh, &ch);  // sin, cos of beta p / 2
    tb.d_lam[j] = j < K_kernel ? 4.0 * sh * sh : 0.0;
    tb.f_lam[j] = (float)tb.d_lam[j];
    // Shears x += t y, y -= s x, x += t y: their product has trace 2 (1 - t s), so it turns by the
    // angle theta' with cos theta' = 1 - t s whatever t and s are (and has determinant one). Rounding
    // t = tan(theta / 2) and s = sin(theta) to FP32 on their own leaves theta' off by about u theta,
    // a phase drift that grows with every step of a long serial recursion. So t is taken within 8
    // ulps of tan(theta / 2) and s next to 2 sin^2(theta / 2) / t, the pair whose exact product
    // (exact in FP64) is closest to 1 - cos(theta) = 2 sin^2(theta / 2): theta' is then right to a
    // small fraction of an ulp, while the map stays within 8 ulps of the rotation.
    float2 shear = make_float2(0.f, 0.f);
    if (j < K_kernel && sh > 0.0) {
      const double target = 2.0 * sh * sh;
      const float t0 = (float)(sh / ch);
      double best = -1.0;
      for (int k = -8; k <= 8; ++k) {
        const float t = __int_as_float(__float_as_int(t0) + k);
        if (!(t > 0.f)) continue;
        const float sc = (float)(target / (double)t);
        for (int q = -1; q <= 1; ++q) {
          const float sv = __int_as_float(__float_as_int(sc) + q);
          const double e = fabs((double)t * (double)sv - target);
          if (best < 0.0 || e < best) {
            best = e;
            shear = make_float2(t, sv);
          }
        }
      }
    }
    tb.f_shear[j] = shear;
  }
  for (int idx = threadIdx.x; idx < K_kernel * 8; idx += blockDim.x) {
    const int j = idx % K_kernel, mm = idx / K_kernel;
    tb.c_pw_chunk[mm][j] = dfc4(power((long long)tb.p0 + j, (long long)items * 32 * (mm + 1)));
  }
  for (int j = threadIdx.x; j < KMAX; j += blockDim.x)
    tb.f_rho[j] = j < K_kernel ? make_float2((float)tb.rho[j].x, (float)tb.rho[j].y) : make_float2(0.f, 0.f);
  for (int idx = threadIdx.x; idx < K_kernel * 17; idx += blockDim.x) {
    const int j = idx % K_kernel, mm = idx / K_kernel;
    const double2 v = power((long long)tb.p0 + j, 512LL * mm);
    tb.f_pw512[mm][j] = make_float2((float)v.x, (float)v.y);
  }
  for (int idx = threadIdx.x; idx < K_kernel * (5 + 32 + 1); idx += blockDim.x) {
    const int j = idx % K_kernel;
    const int q = idx / K_kernel;
    if (q < 5) {
      const double2 v = tb.pw_thr[q][j];
      tb.f_pw_thr[q][j] = make_float2((float)v.x, (float)v.y);
    } else if (q < 37) {
      const double2 v = tb.pw_lane[q - 5][j];
      tb.f_pw_lane_t[j][q - 5] = make_float2((float)v.x, (float)v.y);
      tb.pw_lane_t[j][q - 5] = v;
    } else {
      const double2 v = tb.pw_warp[j];
      const float hx = (float)v.x, hy = (float)v.y;
      tb.f_pwt[0][j] = make_float2(hx, hy);
      tb.f_pwt[1][j] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
    }
  }
  if (threadIdx.x == 0) {
    tb.L = L;
    tb.n0 = J.n0;
    tb.D = L - J.n0;
    tb.items = items;
    tb.alpha = alpha;
    tb.kappa = exp(-2.0 * alpha * (double)L);
    const double gain = exp(alpha * (double)L);
    // E = e^{-alpha^2/(4 gamma)} e^{i omega0 n0}, alpha^2/(4 gamma) = alpha^2 sigma^2 / 2
    const double mag = exp(-0.5 * alpha * alpha * J.sigma * J.sigma);
    double sn, cs;
    sincos(J.omega0 * (double)J.n0, &sn, &cs);
    tb.E = (J.n0 > 0) ? make_double2(mag * cs, mag * sn) : make_double2(1.0, 0.0);
    for (int j = 0; j < KMAX; ++j) {
      const double sg = ((tb.p0 + j) & 1) ? -1.0 : 1.0;  // (-1)^p: c_p - i s_p = (-1)^p V[n + L]
      tb.cM[j] = gain * sg * tb.m[j];
      tb.cL[j] = -gain * sg * tb.l[j];
      tb.f_cM[j] = (float)tb.cM[j];
      tb.f_cL[j] = (float)tb.cL[j];
    }
    if (mult) {
      // V_j(t) = sum_{u = t - 2L}^{t} rho_j^{t - u} x[u] with the lag factor kappa_j = rho_j^{2L};
      // c(omega) + i s(omega) at n (Sec. III-B) is e^{-i omega L} V(n + L), and the Morlet output
      // sum_{p = -P}^{P} a'_p (c + i s)(omega_p) has the complex weights w_j = a'_j e^{-i omega_j L}
      // (a'_0 = a_0, a'_{+-p} = a_p / 2), held as cM_j + i cL_j.
      // The kappa terms: sum_k m_q cos(beta q k) x[n - k] = Re(m_q e^{-i beta q L} V_q(n + L)) with
      // e^{-i beta q L} = (-1)^q, so their weight is the real -kappa_xi (-1)^q m_q on Re V only.
      tb.E = make_double2(1.0, 0.0);
      tb.kappa = 0.0;
      for (int j = 0; j < KMAX; ++j) {
        double wr = 0.0, wi = 0.0, wyr = 0.0, wyi = 0.0;
        if (j < K_kernel && j < n_morlet) {
          const long long q = j - Pm;
          const long long aq = q < 0 ? -q : q;
          const double ap = aq == 0 ? tb.m[0] : 0.5 * tb.m[aq];
          const double2 eL = power(tb.p0 + j, L);
          wr = wyr = ap * eL.x;
          wi = wyi = -ap * eL.y;
        } else if (j < K_kernel && J.kappa_xi != 0.0 && j - n_morlet <= Pm) {
          const long long q = j - n_morlet;
          wr = -J.kappa_xi * ((q & 1) ? -1.0 : 1.0) * tb.m[q];
        }
        tb.cM[j] = wr;
        tb.cL[j] = wi;
        tb.f_cM[j] = (float)wr;
        tb.f_cL[j] = (float)wi;
        tb.f_cMy[j] = (float)wyr;
        tb.f_cLy[j] = (float)wyi;
        const double2 k2 = power(tb.p0 + j, 2 * L);
        tb.f_kapc[j] = j < K_kernel ? make_float2((float)k2.x, (float)k2.y) : make_float2(0.f, 0.f);
      }
    }
    tb.f_E = make_float2((float)tb.E.x, (float)tb.E.y);
    tb.f_kappa = (float)tb.kappa;
  }
}

// Kernel-integral form: two-level table of e^{i pi r / L} = hi[r >> 10] * lo[r & 1023] for the
// per-tile phase anchors (r = (p t) mod 2L is exact; each entry is one FP64 sincospi, rounded once).
__global__ void phase_tables(ScaleTab* tabs, const FitJob* jobs, float2* buf, const long long* poff) {
  const int s = blockIdx.x;
  const long long L = jobs[s].L;
  const long long nhi = (2 * L) / 1024 + 2;
  float2* hi = buf + poff[s];
  float2* lo = hi + nhi;
  for (long long a = threadIdx.x; a < nhi; a += blockDim.x) {
    double sn, cs;
    sincospi((double)((1024 * a) % (2 * L)) / (double)L, &sn, &cs);
    hi[a] = make_float2((float)cs, (float)sn);
  }
  for (int b = threadIdx.x; b < 1024; b += blockDim.x) {
    double sn, cs;
    sincospi((double)b / (double)L, &sn, &cs);
    lo[b] = make_float2((float)cs, (float)sn);
  }
  if (threadIdx.x == 0) {
    tabs[s].ph_hi = hi;
    tabs[s].ph_lo = lo;
  }
}

cudaError_t run_phase_tables(ScaleTab* d_tabs, const FitJob* d_jobs, int n_scales, float2* d_phase,
                             const long long* d_poff, cudaStream_t st) {
  phase_tables<<<n_scales, 256, 0, st>>>(d_tabs, d_jobs, d_phase, d_poff);
  return cudaGetLastError();
}

cudaError_t run_fit(const FitJob* d_jobs, int n_scales, long long max_L, double* d_partial, int nblk,
                    ScaleTab* d_tabs, int K_kernel, int items, int form, cudaStream_t st) {
  dim3 g1(nblk, n_scales);
  fit_partial<<<g1, 256, 0, st>>>(d_jobs, d_partial, nblk);
  fit_solve<<<(n_scales + 31) / 32, 32, 0, st>>>(d_jobs, d_partial, nblk, n_scales, d_tabs);
  return cudaGetLastError();
}

cudaError_t run_tables(ScaleTab* d_tabs, const FitJob* d_jobs, int n_scales, int K_kernel, int items, int form,
                       cudaStream_t st) {
  build_tables<<<n_scales, 256, 0, st>>>(d_tabs, d_jobs, n_scales, K_kernel, items, form);
  return cudaGetLastError();
}

}  // namespace msft
