// The SFT / ASFT window-sum scan (Sec. II-B, II-D, III-A) as one persistent sm_103a kernel.
//
// For every harmonic p_j = p0 + j (beta = pi / L) and every scan position t the kernel keeps the
// window state of the 2L+1 samples x[t-2L .. t]. Two forms are built:
//
//  Kernel-integral form (FORM_KI), the paper's GPU formulation (eqs. kernel, kernelInter,
//  kernelIntZenka): modulate a[t] = x[t] e^{i beta p t}, scan the lagged difference
//  d[t] = a[t] - a[t-2L-1] (its prefix is the window sum u_(2L+1)[t]), then demodulate
//  e^{-i beta p t} u_(2L+1)[t] and combine. Phases are advanced by a fixed step from a per-tile
//  anchor e^{i beta p (t0-1)} looked up from the exact integer (p (t0-1)) mod 2L.
//
//  Rotating form (FORM_RF): the same window sum seen from the harmonic's own frame,
//  V[t] = e^{-i beta p t} u_(2L+1)[t], which obeys the first-order recursion of Sec. II-C (eq. iir1
//  truncated to 2L+1 samples): V[t] = rho V[t-1] + x[t] - rho x[t-2L-1], rho = e^{-i beta p}. The
//  ASFT of Sec. II-D is the same recursion with rho = e^{-alpha - i beta p} and the lagged sample
//  weighted by rho^{2L+1} = kappa rho. A first-order linear recursion is an associative scan over
//  (rho^n, b) pairs, so it runs through the same look-back machinery; no per-sample phase or
//  demodulation is needed, which halves the arithmetic per sample.
//
// Both forms give (c_p - i s_p)[n] = (-1)^p V[n + L] and the direct-method output
// W[n] = sum_p m_p c_p[n] + i l_p s_p[n] (signs folded into the weights cM, cL).
//
// Work decomposition: a row (signal, scale) is cut into segments (work_plan.h); a CTA takes work
// items from a global counter (so every predecessor of a claimed item is already running) and, per
// sub-tile of T = THREADS * ITEMS positions:
//   1. loads x[t] and x[t - 2L - 1] for its ITEMS consecutive positions per thread,
//   2. pass 1: runs the recursion from a zero state -> per-thread aggregate,
//   3. warp-shuffle scan of the aggregates (rotation powers rho^{ITEMS 2^l}),
//   4. warp 0 combines the 8 warp totals (lanes work on (warp, term) pairs in parallel), publishes
//      the tile aggregate and looks back over the segment's earlier tiles (decoupled look-back,
//      bounded waits), or takes the carry of its own previous sub-tile; carries are two-float FP32
//      (compensated), FP32 (plain) or FP64 (FP64 precision),
//   5. pass 2: reruns the recursion from each thread's start state and writes the outputs.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace msft {

enum { FORM_KI = 1, FORM_RF = 2 };
// Output of a position: Morlet direct method W = sum_j cM_j Re V_j + i cL_j Im V_j (complex);
// real (Gaussian smoothing, and the adjoint's planes: sum_j cM_j Re V_j + cL_j Im V_j); or a complex
// combine W = sum_j w_j V_j with w_j = cM_j + i cL_j (multiplication method, non-harmonic terms).
enum { OUT_MORLET = 0, OUT_REAL = 1, OUT_CPLX = 3 };

template <typename R_, typename CV_, int K_, int FORM_, int OUT_, bool ASFT_, int ITEMS_>
struct Cfg {
  using R = R_;
  using V = typename C2<R_>::T;
  using CV = CV_;
  static constexpr int K = K_;
  static constexpr int FORM = FORM_;
  static constexpr int OUT = OUT_;
  static constexpr bool ASFT = ASFT_;
  static constexpr int ITEMS = ITEMS_;
  static constexpr int CH = 1;  // one real input channel
  static constexpr int NT = CH * K_;
  static constexpr int T = THREADS * ITEMS_;
  static constexpr int MINB = (sizeof(R_) == 4 && NT <= 4) ? 3 : (NT <= 8 ? 2 : 1);
  // start states from prefix sums (warp kernel): compensated FP32, real input, rotating form
  static constexpr bool START = std::is_same<CV_, DFC>::value && CH == 1 && FORM_ == FORM_RF && !ASFT_;
  // start states from window sums of Horner tile sums (warp kernel): the damped recursion of the
  // ASFT and the non-harmonic terms of the multiplication method, FP32, real input
  static constexpr bool START_H = ASFT_ && std::is_same<R_, float>::value && CH == 1 && FORM_ == FORM_RF;
  static_assert(FORM_ == FORM_RF || CH == 1, "kernel-integral form is built for real input only");
  static_assert(NT <= 32, "one lane per scanned value in the block phase");
};

template <class C>
struct Smem {
  using R = typename C::R;
  using V = typename C::V;
  using CV = typename C::CV;
  WorkItem wi;
  WorkItem nwi;  // the next work item, loaded while this one runs
  long long work;
  int cur_scale;
  int64_t L, D;
  int32_t p0;
  const float2* ph_hi;
  const float2* ph_lo;
  // staged per scale
  V rho[C::K];
  V pw_thr[5][C::K];
  V pw_lane[32][C::K];
  V pw_wofs_r[8][C::K];
  R cM[C::K], cL[C::K];
  V E;
  R kappa;
  CV pw_wofs_c[8][C::K];
  CV pw_tile_c[33][C::K];
  // per sub-tile
  V wtot[WARPS][C::NT];
  V xw[WARPS][C::NT];
  CV carry[C::NT];
  CV agg[C::NT];
  CV rot[C::NT];
  V base[C::K];
};

// ------------------------------------------------------------------------------------------------
// loads
// ------------------------------------------------------------------------------------------------

// v[i] = p[t + i] if lo <= t + i < hi, else 0. In range and 16-byte aligned: 128-bit loads. In
// range but misaligned by r elements (uniform across a warp in this library's layouts): the aligned
// 128-bit chunks covering the run plus one, shifted by r in registers, provided that superset lies
// inside [0, cap) (cap = elements of the input buffer reachable from p). Otherwise element loads.
template <typename E, int N, int S>
__device__ __forceinline__ void shift_copy(const E* e, E (&v)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) v[i] = e[i + S];
}

template <typename E, int N, int VEC>
__device__ __forceinline__ void shift_in(const int4 (&c)[N / VEC + 1], int r, E (&v)[N]) {
  const E* e = reinterpret_cast<const E*>(c);
  if (r == 1) shift_copy<E, N, 1>(e, v);
  if constexpr (VEC > 2) {
    if (r == 2) shift_copy<E, N, 2>(e, v);
  }
  if constexpr (VEC > 3) {
    if (r == 3) shift_copy<E, N, 3>(e, v);
  }
}

template <typename E, int N>
__device__ __forceinline__ void load_run(const E* __restrict__ p, int64_t t, int64_t lo, int64_t hi,
                                         E (&v)[N], int64_t cap = -1) {
  constexpr int VEC = 16 / sizeof(E);
  if (t >= lo && t + N <= hi) {
    const E* q = p + t;
    const int r = (int)((reinterpret_cast<uintptr_t>(q) & 15) / sizeof(E));
    if (r == 0) {
#pragma unroll
      for (int i = 0; i < N; i += VEC) {
        const int4 u = __ldg(reinterpret_cast<const int4*>(q + i));
        const E* e = reinterpret_cast<const E*>(&u);
#pragma unroll
        for (int j = 0; j < VEC; ++j) v[i + j] = e[j];
      }
      return;
    }
    if constexpr (VEC > 1 && N % VEC == 0) {
      if (cap >= 0 && t - r >= 0 && t - r + N + VEC <= cap) {
        int4 c[N / VEC + 1];
        const int4* a = reinterpret_cast<const int4*>(q - r);
#pragma unroll
        for (int i = 0; i <= N / VEC; ++i) c[i] = __ldg(a + i);
        shift_in<E, N, VEC>(c, r, v);
        return;
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = __ldg(q + i);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int64_t u = t + i;
      v[i] = (u >= lo && u < hi) ? __ldg(p + u) : E{};
    }
  }
}

// 32 bytes of read-only FP32 input in one 256-bit load (sm_100 and later; q 32-byte aligned).
__device__ __forceinline__ void ld_nc_v8(const float* q, float* v) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(q));
}

// load_run for FP32 runs with 256-bit loads: a run of N (a multiple of 8) samples that is in range
// and 32-byte aligned takes N / 8 loads; misaligned by r samples (uniform across a warp in this
// library's layouts), the aligned 32-byte chunks covering it plus one, shifted by r in registers,
// provided that superset lies inside [0, cap). Otherwise as load_run. A lane's run is 64 bytes
// that the warp's 32 lanes read at a 64-byte stride: 32-byte pieces halve the L1 wavefronts of
// 16-byte ones.
template <int N>
__device__ __forceinline__ void load_run_v8(const float* __restrict__ p, int64_t t, int64_t lo, int64_t hi,
                                            float (&v)[N], int64_t cap) {
  static_assert(N % 8 == 0, "runs of whole 32-byte pieces");
  if (t >= lo && t + N <= hi) {
    const float* q = p + t;
    const uintptr_t a = reinterpret_cast<uintptr_t>(q);
    const int r = (int)((a & 31) >> 2);
    if ((a & 31) == 0) {
#pragma unroll
      for (int i = 0; i < N; i += 8) ld_nc_v8(q + i, v + i);
      return;
    }
    if ((a & 3) == 0 && t - r >= 0 && t - r + N + 8 <= cap) {
      float c[N + 8];
#pragma unroll
      for (int i = 0; i < N + 8; i += 8) ld_nc_v8(q - r + i, c + i);
      switch (r) {
        case 1: shift_copy<float, N, 1>(c, v); break;
        case 2: shift_copy<float, N, 2>(c, v); break;
        case 3: shift_copy<float, N, 3>(c, v); break;
        case 4: shift_copy<float, N, 4>(c, v); break;
        case 5: shift_copy<float, N, 5>(c, v); break;
        case 6: shift_copy<float, N, 6>(c, v); break;
        default: shift_copy<float, N, 7>(c, v); break;
      }
      return;
    }
  }
  load_run<float, N>(p, t, lo, hi, v, cap);
}

// Hint: bring elements [a, b) of the n-element buffer at base into L2 with one bulk prefetch (the
// range is shrunk to whole 16-byte granules inside the buffer; nothing is read into registers).
template <typename E>
__device__ __forceinline__ void prefetch_l2(const E* base, int64_t n, int64_t a, int64_t b) {
  if (a < 0) a = 0;
  if (b > n) b = n;
  if (a >= b) return;
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(base + a) + 15) & ~uintptr_t(15);
  const uintptr_t hi = reinterpret_cast<uintptr_t>(base + b) & ~uintptr_t(15);
  if (hi <= lo) return;
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

// Output of item i (position tf + i) at element oo + i. In the common case (all ITEMS positions of
// the lane inside the stored range, 16-byte aligned complex64 output) pairs of items go out as one
// 16-byte streaming store; otherwise each item is checked and stored alone.
template <class C>
__device__ __forceinline__ void store_item(const KParams& P, int64_t oo, int i, typename C::V o, typename C::V prev,
                                           bool all_in, bool in) {
  using R = typename C::R;
  using V = typename C::V;
  if constexpr (C::OUT == OUT_MORLET || C::OUT == OUT_CPLX) {
    V* op = reinterpret_cast<V*>(P.out) + oo;
    if constexpr (sizeof(R) == 4) {
      if (all_in && ((reinterpret_cast<uintptr_t>(op) & 15) == 0)) {
        if (i & 1) __stcs(reinterpret_cast<float4*>(op + (i - 1)), make_float4(prev.x, prev.y, o.x, o.y));
        return;
      }
    }
    if (all_in || in) __stcs(op + i, o);
  } else {
    R* op = reinterpret_cast<R*>(P.out) + oo;
    if (all_in || in) __stcs(op + i, o.x);
  }
}

// ------------------------------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------------------------------

template <class C>
__global__ void __launch_bounds__(THREADS, C::MINB) scan_kernel(const KParams P) {
  using R = typename C::R;
  using V = typename C::V;
  using CV = typename C::CV;
  using CO = CarryOps<CV>;
  constexpr int K = C::K, NT = C::NT, CH = C::CH, ITEMS = C::ITEMS, T = C::T;
  constexpr bool ROT = (C::FORM == FORM_RF);
  // element type of one input sample (real, or complex for the adjoint's two channels)
  using EIn = R;

  __shared__ Smem<C> s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s.cur_scale = -1;
    const long long w = (long long)atomicAdd(P.ticket, 1ull);
    s.work = w;
    if (w < P.n_work) s.wi = P.work[w];
  }
  __syncthreads();

  for (;;) {
    if (s.work >= P.n_work) return;
    const WorkItem wi = s.wi;
    // Independent work items (after the look-back ones) claim the next ticket now, so that its
    // latency hides behind this item; an item that others may wait on is never held unstarted.
    long long next = 0;
    const bool early = s.work >= P.n_chain;
    if (tid == 0 && early) next = (long long)atomicAdd(P.ticket, 1ull);

    if (wi.scale != s.cur_scale) {  // stage this scale's constants (uniform branch)
      const ScaleTab* tb = P.tabs + wi.scale;
      for (int i = tid; i < K; i += THREADS) {
        s.rho[i] = TabR<R>::rho(tb, i);
        s.cM[i] = TabR<R>::cM(tb, i);
        s.cL[i] = TabR<R>::cL(tb, i);
      }
      for (int i = tid; i < 5 * K; i += THREADS) s.pw_thr[i / K][i % K] = conv2<V>(tb->pw_thr[i / K][i % K]);
      for (int i = tid; i < 32 * K; i += THREADS) s.pw_lane[i / K][i % K] = conv2<V>(tb->pw_lane[i / K][i % K]);
      for (int i = tid; i < 8 * K; i += THREADS) {
        s.pw_wofs_r[i / K][i % K] = conv2<V>(tb->pw_wofs[i / K][i % K]);
        s.pw_wofs_c[i / K][i % K] = CO::from_d2(tb->pw_wofs[i / K][i % K]);
      }
      for (int i = tid; i < 33 * K; i += THREADS) s.pw_tile_c[i / K][i % K] = CO::from_d2(tb->pw_tile[i / K][i % K]);
      if (tid == 0) {
        s.E = TabR<R>::E(tb);
        s.kappa = TabR<R>::kappa(tb);
        s.L = tb->L;
        s.D = tb->D;
        s.p0 = tb->p0;
        s.ph_hi = tb->ph_hi;
        s.ph_lo = tb->ph_lo;
      }
      __syncthreads();
      if (tid == 0) s.cur_scale = wi.scale;
    }
    const int64_t L = s.L, D = s.D, Wl = 2 * L + 1;
    const R kap = s.kappa;

    const EIn* __restrict__ xs = reinterpret_cast<const EIn*>(P.x) + wi.x_off;
    const int64_t N = wi.n;
    const int64_t lo = wi.t_dom;  // samples before t_dom count as zero (t_dom >= 0)
    const int64_t t_out = wi.t_out > D ? wi.t_out : D;
    const int64_t t_end = wi.t_end < D + N ? wi.t_end : D + N;
    if (tid < NT) s.carry[tid] = CO::zero();

    for (int sub = 0; sub < wi.n_sub; ++sub) {
      const int64_t t0 = wi.t_a + (int64_t)sub * T;
      const int64_t tf = t0 + (int64_t)tid * ITEMS;  // this thread's first position

      if constexpr (!ROT) {
        // phase anchor e^{i beta p (t0 - 1)} from the exact integer (p (t0 - 1)) mod 2L
        if (tid < K) {
          const long long p = s.p0 + tid, m = 2 * L;
          long long r = (p * (long long)(t0 - 1)) % m;
          if (r < 0) r += m;
          if constexpr (sizeof(R) == 8) {  // FP64 path: the anchor itself in FP64
            double sn, cs;
            sincospi((double)r / (double)L, &sn, &cs);
            s.base[tid] = cmake<R>((R)cs, (R)sn);
          } else {  // two-level table, rounded once per level
            const float2 a = __ldg(s.ph_hi + (r >> 10));
            const float2 b = __ldg(s.ph_lo + (r & 1023));
            const float2 c = cmul(a, b);
            s.base[tid] = cmake<R>((R)c.x, (R)c.y);
          }
        }
        __syncthreads();
      }

      // ---- 1. loads ----
      EIn xa[ITEMS], xl[ITEMS];
      const bool live = (tf + ITEMS > lo && tf < N) || (tf - Wl + ITEMS > lo && tf - Wl < N);
      if (live) {
        load_run<EIn, ITEMS>(xs, tf, lo, N, xa);
        load_run<EIn, ITEMS>(xs, tf - Wl, lo, N, xl, P.n_x - wi.x_off);
      } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) xa[i] = xl[i] = EIn{};
      }

      // thread start phase (kernel-integral form): e^{i beta p (tf - 1)}
      V ph0[ROT ? 1 : K];
      if constexpr (!ROT) {
#pragma unroll
        for (int j = 0; j < K; ++j) ph0[j] = cmul(cmul(s.base[j], s.pw_wofs_r[warp][j]), s.pw_lane[lane][j]);
      }

      // ---- 2. pass 1: per-thread aggregate from a zero state ----
      V B[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) B[v] = V{};
      if (live) {
        if constexpr (ROT) {
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
#pragma unroll
            for (int c = 0; c < CH; ++c) {
              const R xv = reinterpret_cast<const R&>(xa[i]);
              const R xlv = reinterpret_cast<const R&>(xl[i]);
#pragma unroll
              for (int j = 0; j < K; ++j) {
                V& b = B[c * K + j];
                const V r = s.rho[j];
                const R tt = fma(-kap, xlv, b.x);
                const R vr = fma(r.x, tt, fma(-r.y, b.y, xv));
                const R vi = fma(r.y, tt, r.x * b.y);
                b.x = vr;
                b.y = vi;
              }
            }
          }
        } else {
          V ph[K];
#pragma unroll
          for (int j = 0; j < K; ++j) ph[j] = ph0[j];
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
            const R xv = reinterpret_cast<const R&>(xa[i]);
            const R xlv = reinterpret_cast<const R&>(xl[i]);
#pragma unroll
            for (int j = 0; j < K; ++j) {
              const V pn = cmul(ph[j], s.rho[j]);
              B[j].x += fma(xv, pn.x, -xlv * ph[j].x);
              B[j].y += fma(xv, pn.y, -xlv * ph[j].y);
              ph[j] = pn;
            }
          }
        }
      }

      // ---- 3. warp scan of the aggregates (inclusive), exclusive start per lane ----
#pragma unroll
      for (int l = 0; l < 5; ++l) {
        const int o = 1 << l;
#pragma unroll
        for (int v = 0; v < NT; ++v) {
          const V u = shfl_up2(B[v], o);
          if (lane >= o) {
            if constexpr (ROT) B[v] = cfma(s.pw_thr[l][v % K], u, B[v]);
            else {
              B[v].x += u.x;
              B[v].y += u.y;
            }
          }
        }
      }
      if (lane == 31) {
#pragma unroll
        for (int v = 0; v < NT; ++v) s.wtot[warp][v] = B[v];
      }
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        V u = shfl_up2(B[v], 1);
        if (lane == 0) u = V{};
        B[v] = u;
      }
      __syncthreads();

      // ---- 4. block phase: warp 0; lanes take (warp w, term v) pairs, 4 terms per round ----
      if (warp == 0) {
        const int w8 = lane & 7;
        // the tile aggregate is needed for a following sub-tile or for the look-back chain
        const bool need_agg = (sub + 1 < wi.n_sub) || (wi.slot >= 0);
        // a nonzero state enters this sub-tile after an earlier sub-tile or from a predecessor
        const bool has_carry = (sub > 0) || (wi.slot >= 0 && wi.slot != wi.slot_first);
        for (int v0 = 0; v0 < NT; v0 += 4) {
          const int v = v0 + (lane >> 3);
          const bool act = v < NT;
          const int vv = act ? v : 0;
          const V tw = s.wtot[w8][vv];
          // exclusive prefix over the warps (zero entering state), sample precision
          V X = tw;
#pragma unroll
          for (int o = 1; o < 8; o <<= 1) {
            const V u = shfl_up2(X, o);
            if (w8 >= o) {
              if constexpr (ROT) X = cfma(s.pw_wofs_r[o][vv % K], u, X);
              else {
                X.x += u.x;
                X.y += u.y;
              }
            }
          }
          V Xe = shfl_up2(X, 1);
          if (w8 == 0) Xe = V{};
          if (act) s.xw[w8][vv] = Xe;
          if (need_agg) {
            // tile aggregate in carry precision: sum_w rho^{T_w (7 - w)} wtot_w
            CV a = CO::from(tw);
            if constexpr (ROT) a = CO::mul(s.pw_wofs_c[7 - w8][vv % K], a);
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) a = CO::add(a, CO::shfl_xor(a, o));
            if (act && w8 == 0) s.agg[vv] = a;
          }
        }
        __syncwarp();
        const bool lookback = (sub == 0) && (wi.slot >= 0);
        if (lookback) {
          const int64_t slot = wi.slot;
          CV* aggp = reinterpret_cast<CV*>(P.agg);
          CV* inclp = reinterpret_cast<CV*>(P.incl);
          if (slot == wi.slot_first) {
            if (lane < NT) s.carry[lane] = CO::zero();
          } else {
            // publish the aggregate, then look back
            if (lane < NT) {
              st_cg2(aggp + slot * NT + lane, s.agg[lane]);
              __threadfence();
            }
            __syncwarp();
            if (lane == 0) st_release(P.flags + slot, ST_AGG);
            if (lane < NT) {
              s.carry[lane] = CO::zero();
              s.rot[lane] = CO::one();
            }
            __syncwarp();
            int64_t base = slot - 1;
            long long polls = 0;
            bool timed_out = false;
            for (;;) {
              const int64_t j = base - lane;
              const bool valid = (j >= wi.slot_first);
              uint32_t f = ST_INCL;
              bool forced = false;  // a predecessor that never published, after the time limit
              unsigned incl_mask, zero_mask;
              for (;;) {
                f = valid ? ld_acquire(P.flags + j) : ST_INCL;
                forced = timed_out && f == 0;
                if (forced) f = ST_INCL;  // give up: count its state as zero
                incl_mask = __ballot_sync(0xffffffffu, f == ST_INCL);
                zero_mask = __ballot_sync(0xffffffffu, f == 0);
                const int first = incl_mask ? (__ffs(incl_mask) - 1) : 31;
                const unsigned need = (first == 31) ? 0xffffffffu : ((2u << first) - 1u);
                if ((zero_mask & need) == 0) break;
                if (++polls > P.spin_limit) {
                  timed_out = true;
                  if (lane == 0) *reinterpret_cast<volatile int*>(P.err) = DERR_TIMEOUT;
                } else {
                  __nanosleep(64);
                }
              }
              const int first = incl_mask ? (__ffs(incl_mask) - 1) : 32;
              const bool use = (lane <= first) && valid && !forced;
              // sum of predecessor values, lane q rotated by rho^{T q} (times rho^{32 T} per batch)
#pragma unroll
              for (int v = 0; v < NT; ++v) {
                CV val = CO::zero();
                if (use) {
                  const CV* src = (f == ST_INCL) ? inclp : aggp;
                  val = ld_cg2<CV>(src + j * NT + v);
                  if constexpr (ROT) val = CO::mul(s.pw_tile_c[lane][v % K], val);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val = CO::add(val, CO::shfl_xor(val, o));
                if (lane == 0) {
                  if constexpr (ROT) s.carry[v] = CO::add(CO::mul(s.rot[v], val), s.carry[v]);
                  else s.carry[v] = CO::add(s.carry[v], val);
                }
              }
              __syncwarp();
              if (first < 32) break;
              base -= 32;
              if constexpr (ROT) {
                if (lane < NT) s.rot[lane] = CO::mul(s.rot[lane], s.pw_tile_c[32][lane % K]);
              }
              __syncwarp();
            }
          }
          __syncwarp();
          // publish the inclusive state after this tile
          if (lane < NT) {
            CV inc = s.carry[lane];
            if constexpr (ROT) inc = CO::mul(s.pw_tile_c[1][lane % K], inc);
            inc = CO::add(inc, s.agg[lane]);
            st_cg2(inclp + slot * NT + lane, inc);
            __threadfence();
          }
          __syncwarp();
          if (lane == 0) st_release(P.flags + slot, ST_INCL);
        }
        __syncwarp();
        // start state of each warp (sample precision), and the carry into the next sub-tile
        const bool carry_in = has_carry || lookback;
        for (int v0 = 0; carry_in && v0 < NT; v0 += 4) {
          const int v = v0 + (lane >> 3);
          if (v < NT) {
            CV c = s.carry[v];
            if constexpr (ROT) c = CO::mul(s.pw_wofs_c[w8][v % K], c);
            const V cr = conv2<V>(wide2(CO::narrow(c)));
            V xw = s.xw[w8][v];
            xw.x += cr.x;
            xw.y += cr.y;
            s.xw[w8][v] = xw;
          }
        }
        __syncwarp();
        if (lane < NT && sub + 1 < wi.n_sub) {
          CV c = s.carry[lane];
          if constexpr (ROT) c = CO::mul(s.pw_tile_c[1][lane % K], c);
          s.carry[lane] = CO::add(c, s.agg[lane]);
        }
        if (lane == 0 && sub == wi.n_sub - 1) {
          if (!early) next = (long long)atomicAdd(P.ticket, 1ull);
          if (next < P.n_work) s.nwi = P.work[next];
        }
      }
      __syncthreads();

      // ---- 5. pass 2: outputs for positions in [t_out, t_end) ----
      if (tf >= t_end || tf + ITEMS <= t_out) continue;
      V S[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        if constexpr (ROT) S[v] = cfma(s.pw_lane[lane][v % K], s.xw[warp][v], B[v]);
        else {
          S[v].x = s.xw[warp][v].x + B[v].x;
          S[v].y = s.xw[warp][v].y + B[v].y;
        }
      }
      V ph[ROT ? 1 : K];
      if constexpr (!ROT) {
#pragma unroll
        for (int j = 0; j < K; ++j) ph[j] = ph0[j];
      }
      const int64_t oo = wi.out_off - D + tf;  // output element of position tf
      const bool all_in = (tf >= t_out) && (tf + ITEMS <= t_end);
      V prev{};
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        V o = V{};
        if constexpr (ROT) {
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            const R xv = reinterpret_cast<const R&>(xa[i]);
            const R xlv = reinterpret_cast<const R&>(xl[i]);
#pragma unroll
            for (int j = 0; j < K; ++j) {
              V& b = S[c * K + j];
              const V r = s.rho[j];
              const R tt = fma(-kap, xlv, b.x);
              const R vr = fma(r.x, tt, fma(-r.y, b.y, xv));
              const R vi = fma(r.y, tt, r.x * b.y);
              b.x = vr;
              b.y = vi;
              if constexpr (C::OUT == OUT_MORLET) {
                o.x = fma(s.cM[j], vr, o.x);
                o.y = fma(s.cL[j], vi, o.y);
              } else if constexpr (C::OUT == OUT_REAL) {
                o.x = fma(s.cM[j], vr, fma(s.cL[j], vi, o.x));
              } else {
                if (c == 0) o.x = fma(s.cM[j], vr, o.x);
                else o.x = fma(s.cL[j], vi, o.x);
              }
            }
          }
        } else {
          const R xv = reinterpret_cast<const R&>(xa[i]);
          const R xlv = reinterpret_cast<const R&>(xl[i]);
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const V pn = cmul(ph[j], s.rho[j]);
            S[j].x += fma(xv, pn.x, -xlv * ph[j].x);
            S[j].y += fma(xv, pn.y, -xlv * ph[j].y);
            ph[j] = pn;
            const R qx = fma(pn.x, S[j].x, pn.y * S[j].y);  // conj(phase) * window sum
            const R qy = fma(pn.x, S[j].y, -pn.y * S[j].x);
            if constexpr (C::OUT == OUT_MORLET) {
              o.x = fma(s.cM[j], qx, o.x);
              o.y = fma(s.cL[j], qy, o.y);
            } else {
              o.x = fma(s.cM[j], qx, fma(s.cL[j], qy, o.x));
            }
          }
        }
        if constexpr (C::ASFT) o = cmul(o, s.E);
        store_item<C>(P, oo, i, o, prev, all_in, tf + i >= t_out && tf + i < t_end);
        prev = o;
      }
    }
    // hand over to the next work item (its descriptor was loaded during the last block phase)
    __syncthreads();  // everyone is done with this work item's shared state
    if (tid == 0) {
      s.work = next;
      s.wi = s.nwi;
    }
    __syncthreads();
  }
}

}  // namespace msft
