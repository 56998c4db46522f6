// Warp-independent scan for rows whose window is short enough to restart every segment
// ("window" rows). Same arithmetic as scan_kernel.cuh (rotating form), but each warp owns one
// segment of a row and walks it alone, 32 lanes x ITEMS consecutive positions at a time:
//   loads -> pass 1 (recursion from zero) -> warp-shuffle scan -> start state = rho^{ITEMS lane} C + exclusive
//   -> pass 2 (outputs) -> carry C <- rho^{32 ITEMS} C + warp total.
// There is no barrier and no shared memory on the data path, so a stalled warp never holds up the
// others of its CTA. The segment starts from a zero state 2L samples before its first output
// (samples before t_dom count as zero), which keeps the FP32 residue history short; start-state
// items (long windows, compensated FP32) instead begin from the exact state given by the row's
// prefix sums (psum_kernel.cuh). The carry step uses rho^{32 ITEMS} split into two floats so that
// repeated steps do not drift.
#pragma once

#include "psum_kernel.cuh"

namespace msft {

// Table reads in sample precision: FP32 copies for the FP32 kernels, the FP64 tables otherwise.
template <typename V> __device__ __forceinline__ V pw_thr(const ScaleTab* tb, int l, int j);
template <> __device__ __forceinline__ float2 pw_thr<float2>(const ScaleTab* tb, int l, int j) { return __ldg(&tb->f_pw_thr[l][j]); }
template <> __device__ __forceinline__ double2 pw_thr<double2>(const ScaleTab* tb, int l, int j) { return tb->pw_thr[l][j]; }
template <typename V> __device__ __forceinline__ V pw_lane(const ScaleTab* tb, int q, int j);
template <> __device__ __forceinline__ float2 pw_lane<float2>(const ScaleTab* tb, int q, int j) { return __ldg(&tb->f_pw_lane[q][j]); }
template <> __device__ __forceinline__ double2 pw_lane<double2>(const ScaleTab* tb, int q, int j) { return tb->pw_lane[q][j]; }
// rho^{32 ITEMS} as hi (h = 0) + lo (h = 1); for FP64 the whole power in hi and zero in lo
template <typename V> __device__ __forceinline__ V pwt(const ScaleTab* tb, int h, int j);
template <> __device__ __forceinline__ float2 pwt<float2>(const ScaleTab* tb, int h, int j) { return __ldg(&tb->f_pwt[h][j]); }
template <> __device__ __forceinline__ double2 pwt<double2>(const ScaleTab* tb, int h, int j) {
  return h == 0 ? tb->pw_warp[j] : make_double2(0.0, 0.0);
}

template <class C>
__global__ void __launch_bounds__(THREADS, C::MINB) wscan_kernel(const KParams P) {
  using R = typename C::R;
  using V = typename C::V;
  constexpr int K = C::K, NT = C::NT, CH = C::CH, ITEMS = C::ITEMS;
  constexpr int WT = 32 * ITEMS;  // positions per warp-tile
  using EIn = typename std::conditional<CH == 2, V, R>::type;
  const int lane = threadIdx.x & 31;

  long long w = 0;
  if (lane == 0) w = (long long)atomicAdd(P.ticket, 1ull);
  w = __shfl_sync(0xffffffffu, w, 0);
  while (w < P.n_work) {
    const WorkItem wi = P.work[w];
    // claim the next segment now; segments are independent, so holding it is harmless
    long long nxt = 0;
    if (lane == 0) nxt = (long long)atomicAdd(P.ticket, 1ull);

    const ScaleTab* tb = P.tabs + wi.scale;
    const int64_t L = tb->L, D = tb->D, Wl = 2 * L + 1;
    const R kap = (R)tb->kappa;
    V rho[K];
    R cM[K], cL[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      rho[j] = conv2<V>(tb->rho[j]);
      cM[j] = (R)tb->cM[j];
      cL[j] = (C::OUT == OUT_ADJ) ? (R)(-tb->cL[j]) : (R)tb->cL[j];
    }
    const V E = conv2<V>(tb->E);
    const EIn* __restrict__ xs = reinterpret_cast<const EIn*>(P.x) + wi.x_off;
    const int64_t N = wi.n;
    const int64_t lo = wi.t_dom;
    const int64_t t_out = wi.t_out > D ? wi.t_out : D;
    const int64_t t_end = wi.t_end < D + N ? wi.t_end : D + N;

    V Cw[NT];  // state entering the current warp-tile (uniform across lanes)
#pragma unroll
    for (int v = 0; v < NT; ++v) Cw[v] = V{};
    if constexpr (C::START) {
      if (wi.p_row >= 0) start_state<K, ITEMS>(P, wi, tb, rho, lane, Cw);
    }

    for (int k = 0; k < wi.n_sub; ++k) {
      const int64_t tf = wi.t_a + (int64_t)k * WT + (int64_t)lane * ITEMS;
      EIn xa[ITEMS], xl[ITEMS];
      const bool live = (tf + ITEMS > lo && tf < N) || (tf - Wl + ITEMS > lo && tf - Wl < N);
      if (live) {
        load_run<EIn, ITEMS>(xs, tf, lo, N, xa);
        load_run<EIn, ITEMS>(xs, tf - Wl, lo, N, xl, P.n_x - wi.x_off);
      } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) xa[i] = xl[i] = EIn{};
      }
      // pass 1
      V B[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) B[v] = V{};
      if (live) {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
#pragma unroll
          for (int c = 0; c < CH; ++c) {
            R xv, xlv;
            if constexpr (CH == 2) {
              xv = c ? reinterpret_cast<const V&>(xa[i]).y : reinterpret_cast<const V&>(xa[i]).x;
              xlv = c ? reinterpret_cast<const V&>(xl[i]).y : reinterpret_cast<const V&>(xl[i]).x;
            } else {
              xv = reinterpret_cast<const R&>(xa[i]);
              xlv = reinterpret_cast<const R&>(xl[i]);
            }
#pragma unroll
            for (int j = 0; j < K; ++j) {
              V& b = B[c * K + j];
              const R tt = fma(-kap, xlv, b.x);
              const R vr = fma(rho[j].x, tt, fma(-rho[j].y, b.y, xv));
              const R vi = fma(rho[j].y, tt, rho[j].x * b.y);
              b.x = vr;
              b.y = vi;
            }
          }
        }
      }
      // warp scan
#pragma unroll
      for (int l = 0; l < 5; ++l) {
        const int o = 1 << l;
#pragma unroll
        for (int v = 0; v < NT; ++v) {
          const V u = shfl_up2(B[v], o);
          if (lane >= o) B[v] = cfma(pw_thr<V>(tb, l, v % K), u, B[v]);
        }
      }
      V S[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        const V tot = cmake<R>(__shfl_sync(0xffffffffu, B[v].x, 31), __shfl_sync(0xffffffffu, B[v].y, 31));
        V e = shfl_up2(B[v], 1);
        if (lane == 0) e = V{};
        S[v] = cfma(pw_lane<V>(tb, lane, v % K), Cw[v], e);  // state before this lane's first position
        // carry into the next warp-tile: rho^{WT} C + total, with rho^{WT} = hi + lo
        V c = cfma(pwt<V>(tb, 0, v % K), Cw[v], tot);
        Cw[v] = cfma(pwt<V>(tb, 1, v % K), Cw[v], c);
      }
      // pass 2
      if (tf >= t_end || tf + ITEMS <= t_out) continue;
      const int64_t oo = wi.out_off - D + tf;
      const bool all_in = (tf >= t_out) && (tf + ITEMS <= t_end);
      V prev{};
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        V o = V{};
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          R xv, xlv;
          if constexpr (CH == 2) {
            xv = c ? reinterpret_cast<const V&>(xa[i]).y : reinterpret_cast<const V&>(xa[i]).x;
            xlv = c ? reinterpret_cast<const V&>(xl[i]).y : reinterpret_cast<const V&>(xl[i]).x;
          } else {
            xv = reinterpret_cast<const R&>(xa[i]);
            xlv = reinterpret_cast<const R&>(xl[i]);
          }
#pragma unroll
          for (int j = 0; j < K; ++j) {
            V& b = S[c * K + j];
            const R tt = fma(-kap, xlv, b.x);
            const R vr = fma(rho[j].x, tt, fma(-rho[j].y, b.y, xv));
            const R vi = fma(rho[j].y, tt, rho[j].x * b.y);
            b.x = vr;
            b.y = vi;
            if constexpr (C::OUT == OUT_MORLET) {
              o.x = fma(cM[j], vr, o.x);
              o.y = fma(cL[j], vi, o.y);
            } else if constexpr (C::OUT == OUT_REAL) {
              o.x = fma(cM[j], vr, fma(cL[j], vi, o.x));
            } else {
              if (c == 0) o.x = fma(cM[j], vr, o.x);
              else o.x = fma(cL[j], vi, o.x);
            }
          }
        }
        if constexpr (C::ASFT) o = cmul(o, E);
        store_item<C>(P, oo, i, o, prev, all_in, tf + i >= t_out && tf + i < t_end);
        prev = o;
      }
    }
    w = __shfl_sync(0xffffffffu, nxt, 0);
  }
}

}  // namespace msft
