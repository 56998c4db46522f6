// Shared device-side types and helpers of the SFT/ASFT Morlet library (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace msft {

constexpr int KMAX = 12;        // most Fourier terms a plan may use
constexpr int THREADS = 256;    // threads per CTA of the scan kernels
constexpr int WARPS = THREADS / 32;

// Cross-tile status flags (decoupled look-back). 0 = nothing published yet.
constexpr uint32_t ST_AGG = 1;   // the tile's own aggregate is published
constexpr uint32_t ST_INCL = 2;  // the inclusive state after the tile is published

// Device error codes latched in the host-mapped error word.
constexpr int DERR_TIMEOUT = 1;

// ------------------------------------------------------------------------------------------------
// Plan data shared by host and device
// ------------------------------------------------------------------------------------------------

// One (signal, scale) row of the scalogram.
struct ChainDesc {
  int64_t x_off;    // first sample of the signal in x
  int64_t n;        // signal length N
  int64_t out_off;  // first element of the row in the output
  int32_t scale;    // scale index
  int32_t pad;
};

// One unit of work: `n_sub` consecutive sub-tiles of one row, sub-tile s covering scan positions
// t in [t_a + s*T, t_a + (s+1)*T) (the output of position t is n = t - D). Samples before t_dom
// count as zero; outputs are stored for positions in [t_out, t_end). The state entering the work
// item is, in this order of precedence:
//  - p_row >= 0 (start-state items of the warp kernel): computed from the row's lag-free prefix
//    sums P at 512-position tile ends, tile 0 starting at t_grid (psum_kernel.cuh);
//  - slot >= 0: the look-back over status slots [slot_first, slot);
//  - otherwise zero at t_a (the window is recomputed from t_dom).
// Prefix-sum items (psum kernel) use the same record: tiles [t_a, t_a + n_sub * 512) of a row,
// results at prefix index p_row, look-back slot `slot`.
struct WorkItem {
  int64_t x_off;       // the row: first input element, length, first output element, scale
  int64_t n;
  int64_t out_off;
  int32_t scale;
  int32_t chain;
  int32_t n_sub;
  int32_t pad;
  int64_t t_a;
  int64_t t_dom;
  int64_t t_out;
  int64_t t_end;
  int64_t slot;        // status slot of this work item, or -1
  int64_t slot_first;  // status slot of the first work item of the segment
  int64_t p_row;       // prefix-sum index of the row's tile 0 (psum: of the item's first tile), or -1
  int64_t t_grid;      // first position of the row's tile 0 (tiles are 512 positions)
};

// Per-scale constants, all computed on the GPU in FP64 from the fit (tables.cu).
// rho: per-step factor of each harmonic. Rotating form: rho = e^{-alpha} e^{-i beta p}; the window
// state obeys V[t] = rho V[t-1] + x[t] - kappa rho x[t-2L-1]. Kernel-integral form: rho = e^{+i beta p},
// the modulation step. pw_*: powers of rho used by the scans (rotating form only).
struct ScaleTab {
  int64_t L, D;            // half window and output shift (output n reads position n + D)
  int32_t p0, K;           // first harmonic, number of fitted terms
  int32_t n0, items;       // ASFT shift; samples per thread the powers were built for
  double alpha, kappa;     // decay per sample, e^{-2 alpha L}
  double rss, yy;          // fit residual and target energy (sum over the window)
  double2 E;               // output factor (ASFT), 1 otherwise
  double m[KMAX], l[KMAX]; // fitted coefficients of cos / sin (Sec. III-A)
  double cM[KMAX], cL[KMAX];  // combine weights: out.re += cM Re V, out.im += cL Im V
  double2 rho[KMAX];
  double2 pw_thr[5][KMAX];    // rho^{items * 2^l}, l = 0..4
  double2 pw_warp[KMAX];      // rho^{items * 32}
  double2 pw_wofs[8][KMAX];   // rho^{items * 32 * w}
  double2 pw_lane[32][KMAX];  // rho^{items * lane}
  double2 pw_tile[33][KMAX];  // rho^{THREADS * items * q}
  double2 pw_lane_t[KMAX][32];  // pw_lane term-major (the FP64 warp kernel's per-lane reads)
  const float2* ph_hi;        // kernel-integral form: e^{i pi 1024 a / L}, a = 0 .. 2L/1024
  const float2* ph_lo;        // kernel-integral form: e^{i pi b / L}, b = 0 .. 1023
  // FP32 copies for the warp-independent kernel
  float2 f_pw_thr[5][KMAX];   // rho^{items * 2^l}
  float2 f_pw_lane_t[KMAX][32];  // rho^{items * lane}, term-major: the 32 lanes of a warp read one
                                 // term's powers from 256 contiguous bytes (two cache lines)
  float2 f_pwt[2][KMAX];      // rho^{items * 32} as hi + lo
  float4 c_pw_tile[33][KMAX]; // pw_tile as two-float complex (re.hi, re.lo, im.hi, im.lo)
  float4 c_pw_chunk[8][KMAX]; // rho^{32 items (m + 1)}, m = 0..7, two-float complex
  float f_lam[KMAX];          // 4 sin^2(beta p / 2) = |1 - rho|^2 for |rho| = 1 (Reinsch's recurrence)
  double d_lam[KMAX];         // the same in FP64
  float4 c_neg16[32][KMAX];   // rho^{-16 a}, a = 0..31, two-float complex (|rho| = 1)
  float4 c_neg1[16][KMAX];    // rho^{-b}, b = 0..15, two-float complex
  float2 f_shear[KMAX];       // (tan(beta p / 2), sin(beta p)): rho = e^{-i beta p} as three shears
  float2 f_pw512[17][KMAX];   // rho^{512 m}, m = 0..16, FP32
  // FP32 copies of rho, the combine weights, E and kappa (the FP32 kernels never convert from FP64:
  // conversions run on GB300's narrow FP64 pipe)
  float2 f_rho[KMAX];
  float f_cM[KMAX], f_cL[KMAX];
  float2 f_E;
  float f_kappa;
  float2 f_kapc[KMAX];  // multiplication method: rho_j^{2L} per term (non-harmonic, complex)
  // multiplication method: weights of the imaginary part of the combine, out.y += cMy Im V + cLy Re V
  // (equal to cM, cL for the Morlet's complex terms; zero for the kappa terms of the normalised
  // Morlet, whose cosine kernel contributes to the real part only)
  float f_cMy[KMAX], f_cLy[KMAX];
};

// Table reads in the sample precision R (FP32 copies for the FP32 kernels).
template <typename R> struct TabR;
template <> struct TabR<float> {
  __device__ static float2 rho(const ScaleTab* t, int j) { return t->f_rho[j]; }
  __device__ static float cM(const ScaleTab* t, int j) { return t->f_cM[j]; }
  __device__ static float cL(const ScaleTab* t, int j) { return t->f_cL[j]; }
  __device__ static float2 E(const ScaleTab* t) { return t->f_E; }
  __device__ static float kappa(const ScaleTab* t) { return t->f_kappa; }
};
template <> struct TabR<double> {
  __device__ static double2 rho(const ScaleTab* t, int j) { return t->rho[j]; }
  __device__ static double cM(const ScaleTab* t, int j) { return t->cM[j]; }
  __device__ static double cL(const ScaleTab* t, int j) { return t->cL[j]; }
  __device__ static double2 E(const ScaleTab* t) { return t->E; }
  __device__ static double kappa(const ScaleTab* t) { return t->kappa; }
};

struct KParams {
  const void* x;             // input base
  void* out;                 // output base
  const WorkItem* work;
  int64_t n_work;
  const ChainDesc* chains;
  const ScaleTab* tabs;
  uint32_t* flags;           // status flag per slot
  void* agg;                 // per slot: NT complex (carry type)
  void* incl;                // per slot: NT complex (carry type)
  unsigned long long* ticket;
  int* err;                  // host-mapped error word (device view)
  long long spin_limit;
  int64_t n_chain;           // work items [0, n_chain) use the look-back; later ones are independent
  int64_t n_x;               // elements of the input buffer (bounds the widened loads)
  void* pbuf;                // start-state rows: per 512-position tile, K two-float complex prefix
                             // sums (ss_window = 0) or K FP32 complex tile sums (ss_window = 1)
  int ss_window;             // start states from window sums of tile sums instead of prefix sums
  int use_tma;               // warp scan, complex FP32 output: whole warp-tiles leave by TMA stores
  // the output buffer as 2-D tensors of 128-byte rows (32 floats) starting at out + 16 m bytes,
  // m = 0..7, so that a warp-tile starting on any 16-byte boundary is a box of 32 whole rows of one
  // of them (128-byte swizzle)
  CUtensorMap omap[8];
  // lane-chunk scan: the output buffer viewed as rows of one lane chunk each (lmap_c[q] positions,
  // 8 lmap_c[q] bytes; lmap_rows[q] whole rows), boxes of 32 floats x 32 rows, 128-byte swizzle,
  // for up to four chunk lengths (lmap_c[q] = 0: no map)
  CUtensorMap lmap[4];
  int64_t lmap_rows[4];
  int32_t lmap_c[4];
};

// ------------------------------------------------------------------------------------------------
// Small complex helpers
// ------------------------------------------------------------------------------------------------

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename R>
__device__ __forceinline__ typename C2<R>::T cmake(R a, R b) {
  typename C2<R>::T r;
  r.x = a;
  r.y = b;
  return r;
}

// a * b
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// a * b + c
template <typename V>
__device__ __forceinline__ V cfma(V a, V b, V c) {
  V r;
  r.x = fma(a.x, b.x, fma(-a.y, b.y, c.x));
  r.y = fma(a.x, b.y, fma(a.y, b.x, c.y));
  return r;
}

__device__ __forceinline__ float2 to_f2(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(a.x, a.y); }

template <typename V> __device__ __forceinline__ V conv2(double2 a);
template <> __device__ __forceinline__ float2 conv2<float2>(double2 a) { return to_f2(a); }
template <> __device__ __forceinline__ double2 conv2<double2>(double2 a) { return a; }

template <typename V> __device__ __forceinline__ double2 wide2(V a);
template <> __device__ __forceinline__ double2 wide2<float2>(float2 a) { return to_d2(a); }
template <> __device__ __forceinline__ double2 wide2<double2>(double2 a) { return a; }

template <typename V>
__device__ __forceinline__ V shfl_up2(V v, int o) {
  V r;
  r.x = __shfl_up_sync(0xffffffffu, v.x, o);
  r.y = __shfl_up_sync(0xffffffffu, v.y, o);
  return r;
}

template <typename V>
__device__ __forceinline__ V shfl_xor2(V v, int o) {
  V r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, o);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, o);
  return r;
}

// Packed FP32 (sm_100 and later): two independent IEEE single-precision operations per instruction,
// each rounded exactly like the scalar operation. The FP32 scan loops run the Fourier terms in pairs
// (2h, 2h + 1) through them; an odd term count is padded with a zero term (rotation 0, weight 0),
// whose state stays bounded and is never read.
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pk_dup(float a) { return make_float2(a, a); }


template <int K>
struct Pairs {
  static constexpr int H = (K + 1) / 2;
};
// (v[2h], v[2h + 1]), zero past the last term
template <int K>
__device__ __forceinline__ float2 pk_pair(const float (&v)[K], int h) {
  return make_float2(v[2 * h], 2 * h + 1 < K ? v[2 * h + 1] : 0.f);
}

// ITEMS steps of Reinsch's form of the real recurrence of G <- rho G + d from a zero state
// (lam = 4 sin^2(theta / 2)): e <- e + d_i - lam s, s <- s + e, for every term, two terms per
// instruction. Returns e and s after the last step.
template <int K, int ITEMS>
__device__ __forceinline__ void reinsch_pk(const float (&d)[ITEMS], const float (&lam)[K], float (&e)[K],
                                           float (&s)[K]) {
  constexpr int H = Pairs<K>::H;
  float2 nl[H], e2[H], s2[H];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const float2 l = pk_pair<K>(lam, h);
    nl[h] = make_float2(-l.x, -l.y);
    e2[h] = s2[h] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const float2 dd = pk_dup(d[i]);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      e2[h] = pk_fma(nl[h], s2[h], pk_add(e2[h], dd));
      s2[h] = pk_add(s2[h], e2[h]);
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    e[j] = (j & 1) ? e2[j >> 1].y : e2[j >> 1].x;
    s[j] = (j & 1) ? s2[j >> 1].y : s2[j >> 1].x;
  }
}

// ------------------------------------------------------------------------------------------------
// Memory-ordering helpers for the look-back (flags with acquire/release at GPU scope; the values
// are read through L2 with ld.global.cg since L1 is not coherent across SMs).
// ------------------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------------------------------------------------
// Two-float ("double-single") arithmetic for the cross-tile carries of the compensated precision:
// a value is hi + lo with |lo| <= ulp(hi)/2, kept exact by error-free transformations on the FP32
// pipe (GB300's FP64 rate is a small fraction of its FP32 rate). Knuth's TwoSum, Dekker's
// Fast2Sum and an FMA-based TwoProduct.
// ------------------------------------------------------------------------------------------------

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = a + b;
  return DF{s, b - (s - a)};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return fast_two_sum(s, e + a.lo + b.lo);
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// complex two-float
struct DFC {
  DF re, im;
};

__device__ __forceinline__ DFC dfc_add(DFC a, DFC b) { return DFC{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ DFC dfc_mul(DFC a, DFC b) {
  return DFC{df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ DFC dfc_from_d2(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return DFC{DF{rh, (float)(v.x - (double)rh)}, DF{ih, (float)(v.y - (double)ih)}};
}

// Carry arithmetic selected by the carry type: float2 (plain), DFC (compensated), double2 (FP64).
template <typename CV> struct CarryOps;
template <> struct CarryOps<float2> {
  using T = float2;
  __device__ static T zero() { return make_float2(0.f, 0.f); }
  __device__ static T one() { return make_float2(1.f, 0.f); }
  __device__ static T from(float2 a) { return a; }
  __device__ static T from_d2(double2 a) { return make_float2((float)a.x, (float)a.y); }
  __device__ static T add(T a, T b) { return make_float2(a.x + b.x, a.y + b.y); }
  __device__ static T mul(T a, T b) { return cmul(a, b); }
  __device__ static float2 narrow(T a) { return a; }
  __device__ static T shfl_xor(T a, int o) { return shfl_xor2(a, o); }
};
template <> struct CarryOps<double2> {
  using T = double2;
  __device__ static T zero() { return make_double2(0.0, 0.0); }
  __device__ static T one() { return make_double2(1.0, 0.0); }
  __device__ static T from(double2 a) { return a; }
  __device__ static T from_d2(double2 a) { return a; }
  __device__ static T add(T a, T b) { return make_double2(a.x + b.x, a.y + b.y); }
  __device__ static T mul(T a, T b) { return cmul(a, b); }
  __device__ static double2 narrow(T a) { return a; }
  __device__ static T shfl_xor(T a, int o) { return shfl_xor2(a, o); }
};
template <> struct CarryOps<DFC> {
  using T = DFC;
  __device__ static T zero() { return DFC{DF{0.f, 0.f}, DF{0.f, 0.f}}; }
  __device__ static T one() { return DFC{DF{1.f, 0.f}, DF{0.f, 0.f}}; }
  __device__ static T from(float2 a) { return DFC{DF{a.x, 0.f}, DF{a.y, 0.f}}; }
  __device__ static T from_d2(double2 a) { return dfc_from_d2(a); }
  __device__ static T add(T a, T b) { return dfc_add(a, b); }
  __device__ static T mul(T a, T b) { return dfc_mul(a, b); }
  __device__ static float2 narrow(T a) { return make_float2(a.re.hi + a.re.lo, a.im.hi + a.im.lo); }
  __device__ static T shfl_idx(T a, int src) {
    T r;
    r.re.hi = __shfl_sync(0xffffffffu, a.re.hi, src);
    r.re.lo = __shfl_sync(0xffffffffu, a.re.lo, src);
    r.im.hi = __shfl_sync(0xffffffffu, a.im.hi, src);
    r.im.lo = __shfl_sync(0xffffffffu, a.im.lo, src);
    return r;
  }
  __device__ static T shfl_xor(T a, int o) {
    T r;
    r.re.hi = __shfl_xor_sync(0xffffffffu, a.re.hi, o);
    r.re.lo = __shfl_xor_sync(0xffffffffu, a.re.lo, o);
    r.im.hi = __shfl_xor_sync(0xffffffffu, a.im.hi, o);
    r.im.lo = __shfl_xor_sync(0xffffffffu, a.im.lo, o);
    return r;
  }
};

template <typename V> __device__ __forceinline__ V ld_cg2(const V* p);
template <> __device__ __forceinline__ float2 ld_cg2<float2>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ld_cg2<double2>(const double2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ DFC ld_cg2<DFC>(const DFC* p) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  return DFC{DF{v.x, v.y}, DF{v.z, v.w}};
}

__device__ __forceinline__ DFC dfc_from_f4(float4 v) { return DFC{DF{v.x, v.y}, DF{v.z, v.w}}; }
__device__ __forceinline__ DFC dfc_neg(DFC a) { return DFC{df_neg(a.re), df_neg(a.im)}; }

template <typename V> __device__ __forceinline__ void st_cg2(V* p, V v) { __stcg(p, v); }
template <> __device__ __forceinline__ void st_cg2<DFC>(DFC* p, DFC v) {
  __stcg(reinterpret_cast<float4*>(p), make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo));
}

}  // namespace msft
