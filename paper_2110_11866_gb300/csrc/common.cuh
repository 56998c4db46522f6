// Shared device-side types and helpers of the SFT/ASFT Morlet library (sm_103a).
#pragma once

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

// One unit of work: `n_sub` consecutive sub-tiles of one row. Sub-tile k covers scan positions
// t in [D + k*T, D + (k+1)*T) whose outputs are n = t - D. Samples before t_dom count as zero
// (window recomputed from t_dom, no look-back) when slot < 0; otherwise the state entering the
// first sub-tile comes from the look-back over status slots [slot_first, slot).
struct WorkItem {
  int32_t chain;
  int32_t n_sub;
  int64_t k_first;
  int64_t k_out;       // sub-tiles k >= k_out store outputs
  int64_t t_dom;
  int64_t slot;        // status slot of sub-tile k_first, or -1
  int64_t slot_first;  // status slot of the row's first sub-tile
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
  int accumulate;            // adjoint: add to the output instead of overwriting it
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

template <typename V> __device__ __forceinline__ V ld_cg2(const V* p);
template <> __device__ __forceinline__ float2 ld_cg2<float2>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ld_cg2<double2>(const double2* p) { return __ldcg(p); }

}  // namespace msft
