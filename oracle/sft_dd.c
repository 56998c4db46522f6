/*
 * CPU oracle, double-double arithmetic. TEST INFRASTRUCTURE ONLY: called from tests/ and from the
 * cpu_baseline / reference legs of bench.py, never from the CUDA library.
 *
 * oracle_sft_dd:  the kernel-integral SFT of Sec. II-B, step by step in the paper's order,
 *   u[t]      = sum_{s<=t} x[s] e^{i beta p s}                     (eq. kernel)
 *   u_W[t]    = u[t] - u[t - 2L - 1]                               (eq. kernelInter)
 *   c_p[n] - i s_p[n] = e^{-i beta p n} u_W[n + L]                  (the SFT from the kernel integral)
 *   W[n]      = sum_p out_re[p] c_p[n] + i out_im[p] s_p[n]         (direct method, Sec. III-A)
 * The two prefixes u[t] and u[t - 2L - 1] are kept as two running double-double sums (the second
 * trails the first by W = 2L + 1 samples) so that no prefix array is stored. Products x * phase are
 * split exactly with fma (TwoProduct) before they enter the sums. Phases come from the exact
 * integer r = (p t) mod 2L, angle pi r / L.
 *
 * oracle_asft_dd:  the attenuated recursion of Sec. II-D for a window of 2L + 1 samples,
 *   V[t] = rho V[t-1] + x[t] - rho^{2L+1} x[t - 2L - 1],  rho = e^{-alpha - i beta p}
 * (eq. iir1A with the truncation applied inside the recursion, like eq. kernelIntZenka), in
 * double-double, so that V[t] = sum_{s=t-2L}^{t} rho^{t-s} x[s]. The caller combines V.
 *
 * Complex input (for the adjoint) is handled by running the real and imaginary parts as two
 * real inputs.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (contraction off keeps TwoSum exact).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double hi, lo; } dd;

static inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  dd r = {s, e};
  return r;
}

static inline dd dd_add_d(dd a, double b) {
  dd s = two_sum(a.hi, b);
  double lo = s.lo + a.lo;
  return two_sum(s.hi, lo);
}

static inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  double lo = s.lo + a.lo + b.lo;
  return two_sum(s.hi, lo);
}

static inline dd dd_neg(dd a) { dd r = {-a.hi, -a.lo}; return r; }

/* exact product a*b as hi + lo (TwoProduct through fma) added to acc */
static inline dd dd_add_prod(dd acc, double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  acc = dd_add_d(acc, p);
  return dd_add_d(acc, e);
}

/* dd times double, accurate to ~2^-104 relative */
static inline dd dd_mul_d(dd a, double b) {
  double p = a.hi * b;
  double e = fma(a.hi, b, -p);
  e += a.lo * b;
  return two_sum(p, e);
}

static inline double dd_to_d(dd a) { return a.hi + a.lo; }

/*
 * x: n real samples (double). L: half window. p0, K: harmonics p0..p0+K-1.
 * out_re[j], out_im[j]: combine weights, W[n] = sum_j out_re[j] c_j[n] + i out_im[j] s_j[n].
 * W: 2n doubles, interleaved (re, im). Returns 0, or -1 on bad arguments / no memory.
 */
int oracle_sft_dd(const double* x, int64_t n, int64_t L, int32_t p0, int32_t K,
                  const double* out_re, const double* out_im, double* W) {
  if (n < 0 || L < 1 || K < 1 || p0 < 0) return -1;
  const int64_t twoL = 2 * L, Wl = 2 * L + 1;
  double* ct = (double*)malloc(sizeof(double) * (size_t)twoL);
  double* st = (double*)malloc(sizeof(double) * (size_t)twoL);
  dd* ur = (dd*)calloc((size_t)K * 4, sizeof(dd));  /* per term: lead re, lead im, lag re, lag im */
  int64_t* r = (int64_t*)calloc((size_t)K, sizeof(int64_t));
  if (!ct || !st || !ur || !r) { free(ct); free(st); free(ur); free(r); return -1; }
  for (int64_t i = 0; i < twoL; ++i) {      /* e^{i pi i / L}, i = 0..2L-1 */
    double a = M_PI * (double)i / (double)L;
    ct[i] = cos(a);
    st[i] = sin(a);
  }
  memset(W, 0, sizeof(double) * 2 * (size_t)n);
  for (int64_t t = 0; t < n + L; ++t) {
    for (int j = 0; j < K; ++j) {
      const int64_t p = p0 + j;
      /* r_t = (p t) mod 2L kept incrementally; r for t-1 is the phase of x[t-W] (e^{i beta p W} = e^{i beta p}) */
      const int64_t r_prev = (t == 0) ? ((twoL - (p % twoL)) % twoL) : r[j];
      const int64_t r_t = (t == 0) ? 0 : (r[j] + p) % twoL;
      r[j] = r_t;
      dd* u = ur + 4 * j;
      if (t < n) {                                   /* u[t] += x[t] e^{i beta p t} */
        u[0] = dd_add_prod(u[0], x[t], ct[r_t]);
        u[1] = dd_add_prod(u[1], x[t], st[r_t]);
      }
      const int64_t tl = t - Wl;                      /* u[t - W] += x[t-W] e^{i beta p (t-W)} */
      if (tl >= 0 && tl < n) {
        u[2] = dd_add_prod(u[2], x[tl], ct[r_prev]);
        u[3] = dd_add_prod(u[3], x[tl], st[r_prev]);
      }
      if (t >= L) {
        const int64_t nn = t - L;
        const double ur_ = dd_to_d(dd_add(u[0], dd_neg(u[2])));   /* u_W[t] = u[t] - u[t-W] */
        const double ui_ = dd_to_d(dd_add(u[1], dd_neg(u[3])));
        const int64_t rn = (int64_t)(((__int128)p * nn) % twoL); /* e^{-i beta p n} */
        const double c = ct[rn], s = st[rn];
        const double zr = c * ur_ + s * ui_;                     /* z = e^{-i beta p n} u_W = c_p - i s_p */
        const double zi = c * ui_ - s * ur_;
        W[2 * nn] += out_re[j] * zr;                              /* c_p = Re z */
        W[2 * nn + 1] += out_im[j] * (-zi);                       /* s_p = -Im z */
      }
    }
  }
  free(ct); free(st); free(ur); free(r);
  return 0;
}

/*
 * Attenuated recursion (Sec. II-D) over t = 0 .. n + L - 1 - n0 for harmonics p0..p0+K-1 and decay
 * alpha >= 0. For output n the state is read at t = n + L - n0 (the output shift of eq. GsASFT, with
 * the decaying sign reading). Combine: W[n] = E * sum_j (out_re[j] c~_j + i out_im[j] s~_j), where
 * (c~_j - i s~_j)[n - n0] = (-1)^{p_j} e^{alpha L} V_j[n + L - n0] and E = e_re + i e_im.
 */
int oracle_asft_dd(const double* x, int64_t n, int64_t L, int32_t p0, int32_t K, double alpha,
                   int64_t n0, const double* out_re, const double* out_im, double e_re, double e_im,
                   double* W) {
  if (n < 0 || L < 1 || K < 1 || p0 < 0 || alpha < 0 || n0 < 0 || n0 > L) return -1;
  const int64_t twoL = 2 * L, Wl = 2 * L + 1;
  memset(W, 0, sizeof(double) * 2 * (size_t)n);
  double* acc = (double*)calloc(2 * (size_t)n, sizeof(double));
  if (!acc) return -1;
  for (int j = 0; j < K; ++j) {
    const int64_t p = p0 + j;
    const double ang = M_PI * (double)(p % twoL) / (double)L;
    const double dec = exp(-alpha);
    const double rr = dec * cos(ang), ri = -dec * sin(ang);          /* rho = e^{-alpha} e^{-i beta p} */
    /* rho^W = e^{-alpha W} e^{-i beta p (2L+1)} = e^{-alpha W} e^{-i beta p} */
    const double decW = exp(-alpha * (double)Wl);
    const double wr = decW * cos(ang), wi = -decW * sin(ang);
    const double sgn = (p & 1) ? -1.0 : 1.0;
    const double gain = sgn * exp(alpha * (double)L);
    dd vr = {0, 0}, vi = {0, 0};
    for (int64_t t = 0; t < n + L - n0; ++t) {
      /* V <- rho V */
      dd nr = dd_add(dd_mul_d(vr, rr), dd_neg(dd_mul_d(vi, ri)));
      dd ni = dd_add(dd_mul_d(vr, ri), dd_mul_d(vi, rr));
      vr = nr; vi = ni;
      if (t < n) vr = dd_add_d(vr, x[t]);                           /* + x[t] */
      const int64_t tl = t - Wl;
      if (tl >= 0 && tl < n) {                                      /* - rho^W x[t-W] */
        vr = dd_add_prod(vr, -x[tl], wr);
        vi = dd_add_prod(vi, -x[tl], wi);
      }
      const int64_t nn = t - L + n0;
      if (nn >= 0 && nn < n) {
        const double c = gain * dd_to_d(vr);                        /* c~ = (-1)^p e^{alpha L} Re V */
        const double s = -gain * dd_to_d(vi);                       /* s~ = -(-1)^p e^{alpha L} Im V */
        acc[2 * nn] += out_re[j] * c;
        acc[2 * nn + 1] += out_im[j] * s;
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {                                 /* W = E * acc */
    const double a = acc[2 * i], b = acc[2 * i + 1];
    W[2 * i] = e_re * a - e_im * b;
    W[2 * i + 1] = e_re * b + e_im * a;
  }
  free(acc);
  return 0;
}

/*
 * Batched driver for timing: chains (signal i, scale s) run in parallel over OpenMP threads.
 * x_off[i], n_len[i]: signal i in x; L[s], p0[s], out_re/out_im[s*K + j]; W laid out as
 * W[(S * x_off[i] + s * n_len[i] + n)] complex. Returns the number of threads used.
 */
int oracle_sft_dd_batch(const double* x, const int64_t* x_off, const int64_t* n_len, int32_t n_sig,
                        const int64_t* L, const int32_t* p0, int32_t n_scales, int32_t K,
                        const double* out_re, const double* out_im, double* W, int32_t n_threads) {
  int used = 1;
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
  const int64_t n_chain = (int64_t)n_sig * n_scales;
  int err = 0;
#pragma omp parallel
  {
#ifdef _OPENMP
#pragma omp single
    used = omp_get_num_threads();
#endif
#pragma omp for schedule(dynamic, 1)
    for (int64_t c = 0; c < n_chain; ++c) {
      const int64_t i = c / n_scales, s = c % n_scales;
      double* Wc = W + 2 * ((int64_t)n_scales * x_off[i] + s * n_len[i]);
      if (oracle_sft_dd(x + x_off[i], n_len[i], L[s], p0[s], K, out_re + s * K, out_im + s * K, Wc))
        err = 1;
    }
  }
  return err ? -1 : used;
}
