// Warp-independent scan for rows whose window is short enough to restart every segment
// ("window" rows). Same arithmetic as scan_kernel.cuh (rotating form), but each warp owns one
// segment of a row and walks it alone, 32 lanes x ITEMS consecutive positions at a time:
//   loads -> pass 1 (recursion from zero) -> warp-shuffle scan -> start state = rho^{ITEMS lane} C + exclusive
//   -> pass 2 (outputs) -> carry C <- rho^{32 ITEMS} C + warp total.
// There is no CTA barrier: a warp's only shared memory is its own 4 KB output staging tile (whole
// warp-tiles leave it by one TMA tensor store), so a stalled warp never holds up the others of its
// CTA. The segment starts from a zero state 2L samples before its first output
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
template <> __device__ __forceinline__ float2 pw_lane<float2>(const ScaleTab* tb, int q, int j) { return __ldg(&tb->f_pw_lane_t[j][q]); }
template <> __device__ __forceinline__ double2 pw_lane<double2>(const ScaleTab* tb, int q, int j) { return tb->pw_lane_t[j][q]; }
// rho^{32 ITEMS} as hi (h = 0) + lo (h = 1); for FP64 the whole power in hi and zero in lo
template <typename V> __device__ __forceinline__ V pwt(const ScaleTab* tb, int h, int j);
template <> __device__ __forceinline__ float2 pwt<float2>(const ScaleTab* tb, int h, int j) { return __ldg(&tb->f_pwt[h][j]); }
template <> __device__ __forceinline__ double2 pwt<double2>(const ScaleTab* tb, int h, int j) {
  return h == 0 ? tb->pw_warp[j] : make_double2(0.0, 0.0);
}

// One position of the recursion V <- rho (V - kappa xl) + x, for every term of every channel, and
// (OUT) the output combine. Returns the output of the position. (ASFT form.)
template <class C, bool OUT>
__device__ __forceinline__ typename C::V step(typename C::V (&S)[C::NT], const typename C::V (&rho)[C::K],
                                              const typename C::R (&cM)[C::K], const typename C::R (&cL)[C::K],
                                              typename C::R kap, const typename C::R (&xv)[C::CH],
                                              const typename C::R (&xlv)[C::CH],
                                              const typename C::V (&kapc)[C::OUT == OUT_CPLX ? C::K : 1]) {
  using R = typename C::R;
  using V = typename C::V;
  V o = V{};
#pragma unroll
  for (int c = 0; c < C::CH; ++c) {
#pragma unroll
    for (int j = 0; j < C::K; ++j) {
      V& b = S[c * C::K + j];
      R vr, vi;
      if constexpr (C::OUT == OUT_CPLX) {
        // V <- rho (V - kappa_j x_lag) + x with the complex kappa_j = rho_j^{2L} (non-harmonic)
        const R tr = fma(-kapc[j].x, xlv[c], b.x);
        const R ti = fma(-kapc[j].y, xlv[c], b.y);
        vr = fma(rho[j].x, tr, fma(-rho[j].y, ti, xv[c]));
        vi = fma(rho[j].y, tr, rho[j].x * ti);
      } else {
        const R tt = fma(-kap, xlv[c], b.x);
        vr = fma(rho[j].x, tt, fma(-rho[j].y, b.y, xv[c]));
        vi = fma(rho[j].y, tt, rho[j].x * b.y);
      }
      b.x = vr;
      b.y = vi;
      if constexpr (OUT) {
        if constexpr (C::OUT == OUT_CPLX) {
          o.x = fma(cM[j], vr, fma(-cL[j], vi, o.x));
          o.y = fma(cM[j], vi, fma(cL[j], vr, o.y));
        } else if constexpr (C::OUT == OUT_MORLET) {
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
  }
  return o;
}

// SFT form. With rho^{2L} = 1 the window state splits as V(t) = G(t) + x[t - 2L], where G, the sum
// over the 2L samples x[t-2L+1 .. t], obeys G <- rho G + d with the real input d = x[t] - x[t - 2L]
// shared by all terms. One position of that recursion and (OUT) the combine of V; cx = sum_j cM_j
// carries the x[t - 2L] part of Re V (channel 0).
template <class C, bool OUT>
__device__ __forceinline__ typename C::V step_g(typename C::V (&S)[C::NT], const typename C::V (&rho)[C::K],
                                                const typename C::R (&cM)[C::K], const typename C::R (&cL)[C::K],
                                                typename C::R cx, const typename C::R (&d)[C::CH], typename C::R xg0) {
  using R = typename C::R;
  using V = typename C::V;
  V o = V{};
#pragma unroll
  for (int c = 0; c < C::CH; ++c) {
#pragma unroll
    for (int j = 0; j < C::K; ++j) {
      V& b = S[c * C::K + j];
      const R vr = fma(rho[j].x, b.x, fma(-rho[j].y, b.y, d[c]));
      const R vi = fma(rho[j].y, b.x, rho[j].x * b.y);
      b.x = vr;
      b.y = vi;
      if constexpr (OUT) {
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
  }
  if constexpr (OUT) o.x = fma(cx, xg0, o.x);
  return o;
}

template <class C, typename EIn>
__device__ __forceinline__ void split_in(const EIn& a, const EIn& l, typename C::R (&xv)[C::CH],
                                         typename C::R (&xlv)[C::CH]) {
  xv[0] = a;
  xlv[0] = l;
}

// One warp-tile of complex FP32 outputs (32 staged rows of 128 bytes at shared address sa, in the
// 128-byte swizzle) to the output bytes [ofs, ofs + 4096), ofs a multiple of 16, by one TMA tensor
// store of the map whose rows start at that offset modulo 128. The lanes' generic-proxy writes of
// the rows are made visible to the async proxy first; lane 0 issues and commits the store.
__device__ __forceinline__ void tma_store_tile(const KParams& P, uint64_t ofs, uint32_t sa, int lane) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    const int m = (int)((ofs >> 4) & 7);
    const int y = (int)((ofs - 16 * (uint64_t)m) >> 7);
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(&P.omap[m])),
                 "r"(0), "r"(y), "r"(sa)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
}

template <class C>
__global__ void __launch_bounds__(THREADS, C::MINB) wscan_kernel(const __grid_constant__ KParams P) {
  using R = typename C::R;
  using V = typename C::V;
  constexpr int K = C::K, NT = C::NT, CH = C::CH, ITEMS = C::ITEMS;
  constexpr int WT = 32 * ITEMS;  // positions per warp-tile
  // SFT (|rho| = 1, rho^{2L} = 1): the G form above, and a warp scan in the frame of the tile start,
  // where combining two lanes is a plain sum. The damped ASFT keeps the V recursion and the
  // multiplicative scan (rho^{-n} would amplify).
  constexpr bool GF = !C::ASFT;
  // FP32 real input: the per-position loops run the terms in pairs (packed FP32)
  constexpr bool PK = GF && std::is_same<R, float>::value && CH == 1;
  constexpr bool PKM = PK && C::OUT == OUT_MORLET;
  constexpr bool PKR = PK && C::OUT == OUT_REAL;  // real output: both parts folded into one sum
  constexpr bool PKO = PKM || PKR;
  // FP32 ASFT and multiplication method with real input: the recursion V <- rho (V - kappa x_lag) + x
  // (kappa real, or complex per term for the multiplication method) in term pairs
  constexpr bool APK = C::ASFT && std::is_same<R, float>::value && CH == 1 &&
                       (C::OUT == OUT_MORLET || C::OUT == OUT_REAL || C::OUT == OUT_CPLX);
  constexpr bool APC = APK && C::OUT == OUT_CPLX;
  // The ASFT (real kappa = rho^{2L}, shared by every term) runs on U = V - kappa x[t - 2L], which
  // obeys U <- rho U + (x[t] - kappa x[t - 2L]): the window of the last 2L samples, with a real
  // driving term shared by every term (the SFT's form with a damped rho), so that a term pair takes
  // four packed operations per position instead of five. Re V = Re U + kappa x[t - 2L] in the combine.
  constexpr bool AU = APK && !APC;
  constexpr bool V8 = PK || APK;  // 256-bit loads of the FP32 input runs
  constexpr int H = Pairs<K>::H;
  using EIn = R;
  const int lane = threadIdx.x & 31;

  // Work items are claimed two ahead, and the record of the next one is prefetched into L1 while the
  // current one runs, so an item starts without waiting on the work counter. Items are independent,
  // so holding them is harmless.
  long long w = 0, w1 = 0;
  if (lane == 0) {
    w = (long long)atomicAdd(P.ticket, 1ull);
    w1 = (long long)atomicAdd(P.ticket, 1ull);
  }
  w = __shfl_sync(0xffffffffu, w, 0);
  w1 = __shfl_sync(0xffffffffu, w1, 0);
  bool tma_pending = false;  // a TMA store of this warp's staging tile may still be reading it
  V carry{};                 // odd tiles: the last output of the warp's previous tile
  while (w < P.n_work) {
    const WorkItem wi = P.work[w];
    long long w2 = 0;
    if (lane == 0) w2 = (long long)atomicAdd(P.ticket, 1ull);
    if (w1 < P.n_work && lane < (int)(sizeof(WorkItem) + 127) / 128)
      asm volatile("prefetch.global.L1 [%0];" ::"l"(reinterpret_cast<const char*>(P.work + w1) + 128 * lane));

    const ScaleTab* tb = P.tabs + wi.scale;
    const int64_t L = tb->L, D = tb->D;
    const int64_t Wl = (GF || AU) ? 2 * L : 2 * L + 1;  // lag of the second input stream
    const R kap = TabR<R>::kappa(tb);
    V kapc[C::OUT == OUT_CPLX ? K : 1];  // multiplication method: complex lag factor per term
#pragma unroll
    for (int j = 0; j < (C::OUT == OUT_CPLX ? K : 1); ++j)
      kapc[j] = (C::OUT == OUT_CPLX) ? cmake<R>((R)tb->f_kapc[j].x, (R)tb->f_kapc[j].y) : V{};
    V rho[K], pn[GF ? K : 1];
    R cM[K], cL[K];
    R cx = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      rho[j] = TabR<R>::rho(tb, j);
      cM[j] = TabR<R>::cM(tb, j);
      cL[j] = TabR<R>::cL(tb, j);
      cx += cM[j];
      if constexpr (GF) {  // conj(rho^{ITEMS (lane + 1)}) = rho^{-ITEMS (lane + 1)}
        const V q = cmul(pw_lane<V>(tb, lane, j), pw_thr<V>(tb, 0, j));
        pn[j].x = q.x;
        pn[j].y = -q.y;
      }
    }
    // packed constants of the FP32 Morlet and real-output loops (term pairs; a padded term has
    // rho = 0, weight 0)
    float2 rx2[H], ry2[H], nry2[H], cm2[H], cl2[H];
    if constexpr (PKO || APK) {
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const bool two = 2 * h + 1 < K;
        const V r0 = rho[2 * h], r1 = two ? rho[2 * h + 1] : V{};
        rx2[h] = make_float2(r0.x, r1.x);
        ry2[h] = make_float2(r0.y, r1.y);
        nry2[h] = make_float2(-r0.y, -r1.y);
        cm2[h] = make_float2(cM[2 * h], two ? cM[2 * h + 1] : 0.f);
        cl2[h] = make_float2(cL[2 * h], two ? cL[2 * h + 1] : 0.f);
      }
    }
    // multiplication method, in pairs: -kappa_j, and the weights of the imaginary part of the combine
    float2 nkr2[APC ? H : 1], nki2[APC ? H : 1], cmy2[APC ? H : 1], cly2[APC ? H : 1];
    if constexpr (APC) {
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const bool two = 2 * h + 1 < K;
        nkr2[h] = make_float2(-kapc[2 * h].x, two ? -kapc[2 * h + 1].x : 0.f);
        nki2[h] = make_float2(-kapc[2 * h].y, two ? -kapc[2 * h + 1].y : 0.f);
        cmy2[h] = make_float2(__ldg(&tb->f_cMy[2 * h]), two ? __ldg(&tb->f_cMy[2 * h + 1]) : 0.f);
        cly2[h] = make_float2(__ldg(&tb->f_cLy[2 * h]), two ? __ldg(&tb->f_cLy[2 * h + 1]) : 0.f);
      }
    }
    const V E = TabR<R>::E(tb);
    const R cxk = cx * kap;  // U form: the kappa x[t - 2L] part of Re V, summed over the terms
    const EIn* __restrict__ xs = reinterpret_cast<const EIn*>(P.x) + wi.x_off;
    const int64_t N = wi.n;
    const int64_t lo = wi.t_dom;
    const int64_t t_out = wi.t_out > D ? wi.t_out : D;
    const int64_t t_end = wi.t_end < D + N ? wi.t_end : D + N;

    V Cw[NT];  // state entering the current warp-tile (uniform across lanes)
#pragma unroll
    for (int v = 0; v < NT; ++v) Cw[v] = V{};
    if constexpr (C::START) {
      if (wi.p_row >= 0) {
        if (P.ss_window) start_state_window<K, ITEMS>(P, wi, tb, rho, lane, Cw);
        else start_state<K, ITEMS>(P, wi, tb, rho, lane, Cw);
      }
    } else if constexpr (C::START_H) {
      if (wi.p_row >= 0) start_state_window<K, ITEMS, true>(P, wi, tb, rho, lane, Cw);
    }
    if constexpr (AU) {
      // V(b - 1) -> U(b - 1) = V(b - 1) - kappa x[b - 1 - 2L], b = the item's first position (zero
      // for a window segment: its state and the samples before its restart are zero)
      const int64_t u = wi.t_a - 1 - 2 * L;
      const R xu = (u >= lo && u < N) ? xs[u] : R(0);
#pragma unroll
      for (int v = 0; v < NT; ++v) Cw[v].x = fma(-kap, xu, Cw[v].x);
    }

    for (int k = 0; k < wi.n_sub; ++k) {
      const int64_t tf = wi.t_a + (int64_t)k * WT + (int64_t)lane * ITEMS;
      if constexpr (PKM) {
        // SFT Morlet, FP32 input: an L2 prefetch of the input run two warp-tiles ahead (one bulk prefetch
        // of 2 KB, issued by lane 0 through a predicate inside the asm, which keeps a divergent
        // branch out of the loop). Measured on the full scalogram: one tile ahead -1.1 %, two
        // ahead +0.6 %; for the damped recursions -3 % and for real output -4 %, so they have none.
        const int64_t a = wi.x_off + wi.t_a + (int64_t)(k + 2) * WT;
        const bool ok = k + 2 < wi.n_sub && a >= 4 && a + WT <= P.n_x;  // (rounded down: stays inside)
        const uintptr_t pa = reinterpret_cast<uintptr_t>(reinterpret_cast<const float*>(P.x) + a) & ~uintptr_t(15);
        asm volatile("{ .reg .pred p; setp.ne.u32 p, %1, 0; @p cp.async.bulk.prefetch.L2.global [%0], 2048; }" ::"l"(pa),
                     "r"((unsigned)(ok && lane == 0)));
      }
      EIn xa[ITEMS], xl[ITEMS];
      const bool live = (tf + ITEMS > lo && tf < N) || (tf - Wl + ITEMS > lo && tf - Wl < N);
      if (live) {
        if constexpr (V8) {
          load_run_v8<ITEMS>(xs, tf, lo, N, xa, P.n_x - wi.x_off);
          load_run_v8<ITEMS>(xs, tf - Wl, lo, N, xl, P.n_x - wi.x_off);
        } else {
          load_run<EIn, ITEMS>(xs, tf, lo, N, xa);
          load_run<EIn, ITEMS>(xs, tf - Wl, lo, N, xl, P.n_x - wi.x_off);
        }
      } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) xa[i] = xl[i] = EIn{};
      }
      // pass 1: the lane's aggregate from a zero state
      V B[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) B[v] = V{};
      if (live) {
        if constexpr (GF) {
          // 16 steps of G <- rho G + d from zero as the real second-order recurrence in Reinsch's
          // form (rho = e^{-i theta}, lam = 4 sin^2(theta / 2)):
          //     e_i = e_{i-1} + d_i - lam s_{i-1},  s_i = s_{i-1} + e_i,
          // then G = (e_15 + (lam / 2) s_14) - i sin(theta) s_14 with s_14 = s_15 - e_15.
          R sv[NT], ev[NT], lam[K];
#pragma unroll
          for (int j = 0; j < K; ++j) {
            if constexpr (sizeof(R) == 4) lam[j] = __ldg(&tb->f_lam[j]);
            else lam[j] = tb->d_lam[j];
          }
          if constexpr (PK) {
            float d[ITEMS];
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) d[i] = xa[i] - xl[i];
            reinsch_pk<K, ITEMS>(d, lam, ev, sv);
          } else {
#pragma unroll
            for (int v = 0; v < NT; ++v) sv[v] = ev[v] = R(0);
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
              R xv[CH], xgv[CH];
              split_in<C>(xa[i], xl[i], xv, xgv);
#pragma unroll
              for (int c = 0; c < CH; ++c) {
                const R dd = xv[c] - xgv[c];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                  const int v = c * K + j;
                  ev[v] = fma(-lam[j], sv[v], ev[v] + dd);
                  sv[v] += ev[v];
                }
              }
            }
          }
#pragma unroll
          for (int v = 0; v < NT; ++v) {
            const R s14 = sv[v] - ev[v];
            B[v].x = fma(R(0.5) * lam[v % K], s14, ev[v]);
            if constexpr (PKO) B[v].y = ((v & 1) ? ry2[v >> 1].y : ry2[v >> 1].x) * s14;
            else B[v].y = rho[v % K].y * s14;
          }
        } else if constexpr (AU) {
          // U <- rho U + d from zero, d = x[t] - kappa x[t - 2L], two terms per instruction, as the
          // real second-order recurrence in Reinsch's form for a damped rotation (rho = r e^{-i theta},
          // r = |rho| = e^{-alpha} for every term, lam = 4 sin^2(theta / 2)):
          //     e_i = r e_{i-1} + d_i - r lam s_{i-1},  s_i = r s_{i-1} + e_i,
          // then U = (e_15 + (r lam / 2) s_14) + i Im(rho) s_14: three operations per position and
          // term pair instead of four.
          const float r = sqrtf(fmaf(rho[0].x, rho[0].x, rho[0].y * rho[0].y));
          const float2 r2 = pk_dup(r);
          float2 nl2[H], e2[H], s2[H];
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const float l0 = __ldg(&tb->f_lam[2 * h]), l1 = 2 * h + 1 < K ? __ldg(&tb->f_lam[2 * h + 1]) : 0.f;
            nl2[h] = make_float2(-r * l0, -r * l1);
            e2[h] = s2[h] = make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
            const float2 d2 = pk_dup(fmaf(-kap, xl[i], xa[i]));
#pragma unroll
            for (int h = 0; h < H; ++h) {
              e2[h] = pk_fma(nl2[h], s2[h], pk_fma(r2, e2[h], d2));
              if (i + 1 < ITEMS) s2[h] = pk_fma(r2, s2[h], e2[h]);  // the last step keeps s_14
            }
          }
#pragma unroll
          for (int v = 0; v < NT; ++v) {
            const int h = v >> 1;
            const float e = (v & 1) ? e2[h].y : e2[h].x, s14 = (v & 1) ? s2[h].y : s2[h].x;
            const float nl = (v & 1) ? nl2[h].y : nl2[h].x, ry = (v & 1) ? ry2[h].y : ry2[h].x;
            B[v] = cmake<R>(fmaf(-0.5f * nl, s14, e), ry * s14);
          }
        } else if constexpr (APK) {
          // the damped recursion from zero, two terms per instruction (the scalar step's operations
          // in the same order)
          float2 X2[H], Y2[H];
#pragma unroll
          for (int h = 0; h < H; ++h) X2[h] = Y2[h] = make_float2(0.f, 0.f);
          const float2 nk2 = pk_dup(-kap);
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
            const float2 xv2 = pk_dup(xa[i]), xl2 = pk_dup(xl[i]);
#pragma unroll
            for (int h = 0; h < H; ++h) {
              float2 tt, ti;
              if constexpr (APC) {
                tt = pk_fma(nkr2[h], xl2, X2[h]);
                ti = pk_fma(nki2[h], xl2, Y2[h]);
              } else {
                tt = pk_fma(nk2, xl2, X2[h]);
                ti = Y2[h];
              }
              const float2 vr = pk_fma(rx2[h], tt, pk_fma(nry2[h], ti, xv2));
              Y2[h] = pk_fma(ry2[h], tt, pk_mul(rx2[h], ti));
              X2[h] = vr;
            }
          }
#pragma unroll
          for (int v = 0; v < NT; ++v)
            B[v] = (v & 1) ? cmake<R>(X2[v >> 1].y, Y2[v >> 1].y) : cmake<R>(X2[v >> 1].x, Y2[v >> 1].x);
        } else {
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
            R xv[CH], xlv[CH];
            split_in<C>(xa[i], xl[i], xv, xlv);
            step<C, false>(B, rho, cM, cL, kap, xv, xlv, kapc);
          }
        }
      }
      // warp scan -> S: state before the lane's first position; Cw advances by one warp-tile
      V S[NT];
      if constexpr (GF) {
        // B'_l = rho^{-ITEMS (l+1)} B_l; the state before lane l is rho^{ITEMS l} (Cw + sum_{l'<l} B'_l')
        // and the state after the tile rho^{WT} (Cw + sum_l B'_l).
#pragma unroll
        for (int v = 0; v < NT; ++v) B[v] = cmul(pn[v % K], B[v]);
#pragma unroll
        for (int l = 0; l < 5; ++l) {
          const int o = 1 << l;
#pragma unroll
          for (int v = 0; v < NT; ++v) {
            const V u = shfl_up2(B[v], o);
            if (lane >= o) {
              B[v].x += u.x;
              B[v].y += u.y;
            }
          }
        }
#pragma unroll
        for (int v = 0; v < NT; ++v) {
          const V tot = cmake<R>(__shfl_sync(0xffffffffu, B[v].x, 31), __shfl_sync(0xffffffffu, B[v].y, 31));
          V e = shfl_up2(B[v], 1);
          if (lane == 0) e = V{};
          S[v] = cmul(pw_lane<V>(tb, lane, v % K), cmake<R>(Cw[v].x + e.x, Cw[v].y + e.y));
          // rho^{WT} = hi + lo (two floats) so that repeated steps do not drift
          const V c = cmake<R>(Cw[v].x + tot.x, Cw[v].y + tot.y);
          Cw[v] = cfma(pwt<V>(tb, 0, v % K), c, cmul(pwt<V>(tb, 1, v % K), c));
        }
      } else {
#pragma unroll
        for (int l = 0; l < 5; ++l) {
          const int o = 1 << l;
#pragma unroll
          for (int v = 0; v < NT; ++v) {
            const V u = shfl_up2(B[v], o);
            if (lane >= o) B[v] = cfma(pw_thr<V>(tb, l, v % K), u, B[v]);
          }
        }
#pragma unroll
        for (int v = 0; v < NT; ++v) {
          const V tot = cmake<R>(__shfl_sync(0xffffffffu, B[v].x, 31), __shfl_sync(0xffffffffu, B[v].y, 31));
          V e = shfl_up2(B[v], 1);
          if (lane == 0) e = V{};
          S[v] = cfma(pw_lane<V>(tb, lane, v % K), Cw[v], e);
          V c = cfma(pwt<V>(tb, 0, v % K), Cw[v], tot);
          Cw[v] = cfma(pwt<V>(tb, 1, v % K), Cw[v], c);
        }
      }
      // pass 2: outputs for positions in [t_out, t_end)
      // packed state (Morlet or real output): X = (Re G_2h, Re G_2h+1), Y likewise
      float2 X2[H], Y2[H];
      if constexpr (PKO || APK) {
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const V s0 = S[2 * h], s1 = 2 * h + 1 < K ? S[2 * h + 1] : V{};
          X2[h] = make_float2(s0.x, s1.x);
          Y2[h] = make_float2(s0.y, s1.y);
        }
      }
      auto one = [&](int i) -> V {
        if constexpr (PKM) {
          // G <- rho G + d and the combine, two terms per instruction
          const float2 dd = pk_dup(xa[i] - xl[i]);
          float2 ox = make_float2(0.f, 0.f), oy = make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const float2 vr = pk_fma(rx2[h], X2[h], pk_fma(nry2[h], Y2[h], dd));
            const float2 vi = pk_fma(ry2[h], X2[h], pk_mul(rx2[h], Y2[h]));
            X2[h] = vr;
            Y2[h] = vi;
            ox = pk_fma(cm2[h], vr, ox);
            oy = pk_fma(cl2[h], vi, oy);
          }
          return cmake<R>(fma(cx, xl[i], ox.x + ox.y), oy.x + oy.y);
        } else if constexpr (PKR) {
          // real output: sum_j cM_j Re V_j + cL_j Im V_j, two terms per instruction
          const float2 dd = pk_dup(xa[i] - xl[i]);
          float2 ox = make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const float2 vr = pk_fma(rx2[h], X2[h], pk_fma(nry2[h], Y2[h], dd));
            const float2 vi = pk_fma(ry2[h], X2[h], pk_mul(rx2[h], Y2[h]));
            X2[h] = vr;
            Y2[h] = vi;
            ox = pk_fma(cl2[h], vi, pk_fma(cm2[h], vr, ox));
          }
          return cmake<R>(fma(cx, xl[i], ox.x + ox.y), R(0));
        } else if constexpr (AU) {
          // U <- rho U + d and the combine (Re V = Re U + kappa x[t - 2L]), two terms per
          // instruction, then the ASFT factor E
          const float2 dd = pk_dup(fmaf(-kap, xl[i], xa[i]));
          float2 ox = make_float2(0.f, 0.f), oy = make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < H; ++h) {
            const float2 vr = pk_fma(rx2[h], X2[h], pk_fma(nry2[h], Y2[h], dd));
            const float2 vi = pk_fma(ry2[h], X2[h], pk_mul(rx2[h], Y2[h]));
            X2[h] = vr;
            Y2[h] = vi;
            if constexpr (C::OUT == OUT_MORLET) {
              ox = pk_fma(cm2[h], vr, ox);
              oy = pk_fma(cl2[h], vi, oy);
            } else {
              ox = pk_fma(cl2[h], vi, pk_fma(cm2[h], vr, ox));
            }
          }
          return cmul(cmake<R>(fma(cxk, xl[i], ox.x + ox.y), oy.x + oy.y), E);
        } else if constexpr (APK) {
          // damped recursion and combine, two terms per instruction, then the ASFT factor E
          const float2 xv2 = pk_dup(xa[i]), xl2 = pk_dup(xl[i]), nk2 = pk_dup(-kap);
          float2 ox = make_float2(0.f, 0.f), oy = make_float2(0.f, 0.f), oz = make_float2(0.f, 0.f);
#pragma unroll
          for (int h = 0; h < H; ++h) {
            float2 tt, ti;
            if constexpr (APC) {
              tt = pk_fma(nkr2[h], xl2, X2[h]);
              ti = pk_fma(nki2[h], xl2, Y2[h]);
            } else {
              tt = pk_fma(nk2, xl2, X2[h]);
              ti = Y2[h];
            }
            const float2 vr = pk_fma(rx2[h], tt, pk_fma(nry2[h], ti, xv2));
            const float2 vi = pk_fma(ry2[h], tt, pk_mul(rx2[h], ti));
            X2[h] = vr;
            Y2[h] = vi;
            if constexpr (C::OUT == OUT_MORLET) {
              ox = pk_fma(cm2[h], vr, ox);
              oy = pk_fma(cl2[h], vi, oy);
            } else if constexpr (C::OUT == OUT_REAL) {
              ox = pk_fma(cl2[h], vi, pk_fma(cm2[h], vr, ox));
            } else {  // complex weights w_j = cM_j + i cL_j: Re(w V) + i (cMy Im V + cLy Re V)
              ox = pk_fma(cm2[h], vr, ox);
              oz = pk_fma(cl2[h], vi, oz);
              oy = pk_fma(cmy2[h], vi, pk_fma(cly2[h], vr, oy));
            }
          }
          if constexpr (APC) return cmul(cmake<R>((ox.x + ox.y) - (oz.x + oz.y), oy.x + oy.y), E);
          return cmul(cmake<R>(ox.x + ox.y, oy.x + oy.y), E);
        }
        R xv[CH], xlv[CH];
        split_in<C>(xa[i], xl[i], xv, xlv);
        V o;
        if constexpr (GF) {
          R dd[CH];
#pragma unroll
          for (int c = 0; c < CH; ++c) dd[c] = xv[c] - xlv[c];
          o = step_g<C, true>(S, rho, cM, cL, cx, dd, xlv[0]);
        } else {
          o = step<C, true>(S, rho, cM, cL, kap, xv, xlv, kapc);
        }
        if constexpr (C::ASFT) o = cmul(o, E);
        return o;
      };
      constexpr bool STAGE = ((C::OUT == OUT_MORLET || C::OUT == OUT_CPLX) && sizeof(R) == 4 && ITEMS == 16);
      constexpr bool STAGE_R = (C::OUT == OUT_REAL && sizeof(R) == 4 && ITEMS == 16);
      const int64_t tw = wi.t_a + (int64_t)k * WT;  // first position of the warp-tile
      if (tw >= t_end || tw + WT <= t_out) continue;  // no output in this warp-tile (warp-uniform)
      if constexpr (STAGE) {
        V* ob = reinterpret_cast<V*>(P.out) + (wi.out_off - D + tw);
        const bool full = tw >= t_out && tw + WT <= t_end;
        // The warp's 512 outputs are staged in its 4 KB tile of shared memory: lane l's 128 bytes
        // form row l, and its 16-byte chunk c sits at chunk position c ^ (l & 7) (the TMA unit's
        // 128-byte swizzle), so that the 8 lanes of each quarter-warp writing chunk c cover all 32
        // banks. A whole tile on a 16-byte boundary then leaves as one TMA tensor store of 32 rows;
        // other tiles are stored from the staged rows, masked to [t_out, t_end).
        __shared__ __align__(1024) float4 s_tile[WARPS * 256];
        float4* rows = s_tile + (threadIdx.x >> 5) * 256;
        if (tma_pending) {  // the previous tile's store must have read the staging tile
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          __syncwarp();
          tma_pending = false;
        }
        const uint64_t ofs = (uint64_t)(wi.out_off - D + tw) * sizeof(V);  // bytes from the output base
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(rows);
        // (the swizzle pattern is that of 1024-byte aligned shared addresses)
        const bool tma = P.use_tma && full && (sa & 1023) == 0;
        const bool odd = (ofs & 15) == 8;  // the tile starts on an 8-byte boundary only
        if (tma && odd && tw > t_out && k > 0) {
          // Odd tile: the box starts one output earlier, at the previous warp-tile's last output
          // (computed by this warp and carried; written before, rewritten with the same value), so
          // row l holds outputs 16 l - 1 .. 16 l + 14; the tile's last output, outside the box,
          // is stored by lane 31 itself.
          const V f = one(0);
#pragma unroll
          for (int c = 1; c < ITEMS / 2; ++c) {
            const V a = one(2 * c - 1);
            const V b = one(2 * c);
            rows[lane * 8 + (c ^ (lane & 7))] = make_float4(a.x, a.y, b.x, b.y);
          }
          const V l = one(ITEMS - 1);
          V pv = cmake<R>(__shfl_up_sync(0xffffffffu, l.x, 1), __shfl_up_sync(0xffffffffu, l.y, 1));
          if (lane == 0) pv = carry;
          rows[lane * 8 + (lane & 7)] = make_float4(pv.x, pv.y, f.x, f.y);
          carry = cmake<R>(__shfl_sync(0xffffffffu, l.x, 31), __shfl_sync(0xffffffffu, l.y, 31));
          if (lane == 31) __stcs(ob + (WT - 1), l);
          tma_store_tile(P, ofs - 8, sa, lane);
          tma_pending = true;
          continue;
        }
#pragma unroll
        for (int i = 0; i < ITEMS; i += 2) {
          const V o0 = one(i);
          const V o1 = one(i + 1);
          rows[lane * 8 + ((i / 2) ^ (lane & 7))] = make_float4(o0.x, o0.y, o1.x, o1.y);
        }
        if (tma && !odd) {
          tma_store_tile(P, ofs, sa, lane);
          tma_pending = true;
          continue;
        }
        __syncwarp();
        const int lo_o = (int)(t_out > tw ? t_out - tw : 0);  // stored outputs [lo_o, hi_o)
        const int hi_o = (int)(t_end < tw + WT ? t_end - tw : WT);
        if ((reinterpret_cast<uintptr_t>(ob) & 15) == 0) {
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const int c = 32 * r + lane;  // 16-byte chunk of the tile: outputs 2c, 2c + 1
            const float4 v = rows[(c >> 3) * 8 + ((c & 7) ^ ((c >> 3) & 7))];
            const bool in0 = 2 * c >= lo_o && 2 * c < hi_o, in1 = 2 * c + 1 >= lo_o && 2 * c + 1 < hi_o;
            if (in0 && in1) __stcs(reinterpret_cast<float4*>(ob) + c, v);
            else if (in0) __stcs(ob + 2 * c, make_float2(v.x, v.y));
            else if (in1) __stcs(ob + 2 * c + 1, make_float2(v.z, v.w));
          }
        } else {
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const int o = 32 * r + lane;
            const int row = o >> 4;
            if (o >= lo_o && o < hi_o)
              __stcs(ob + o, reinterpret_cast<const float2*>(rows + row * 8 + (((o & 15) >> 1) ^ (row & 7)))[o & 1]);
          }
          // the tile's last output (row 31, chunk 7 at position 7 ^ 7 = 0) for the next, shifted box
          const float4 e = rows[31 * 8];
          carry = cmake<R>(e.z, e.w);
        }
        __syncwarp();
      } else if constexpr (STAGE_R) {
        float* obr = reinterpret_cast<float*>(P.out) + (wi.out_off - D + tw);
        const int lo_o = (int)(t_out > tw ? t_out - tw : 0);  // stored outputs [lo_o, hi_o)
        const int hi_o = (int)(t_end < tw + WT ? t_end - tw : WT);
        if (lo_o == 0 && hi_o == WT && (reinterpret_cast<uintptr_t>(obr) & 31) == 0) {
          // every output of the tile, 32-byte aligned: each lane writes its 64 bytes as two
          // whole-sector 256-bit stores
          float* op = obr + lane * ITEMS;
#pragma unroll
          for (int i = 0; i < ITEMS; i += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = one(i + u).x;
            asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(op + i), "f"(v[0]),
                         "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                         : "memory");
          }
          continue;
        }
        // Otherwise through this warp's shared rows (17 floats per lane: conflict-free writes), so
        // that each store instruction writes 128 contiguous bytes; positions outside
        // [t_out, t_end) are masked.
        __shared__ float s_outr[WARPS * 32 * 17];
        float* rows = s_outr + (threadIdx.x >> 5) * (32 * 17);
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) rows[lane * 17 + i] = one(i).x;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
          const int o = 32 * r + lane;
          if (o >= lo_o && o < hi_o) __stcs(obr + o, rows[(o >> 4) * 17 + (o & 15)]);
        }
        __syncwarp();
      } else {
        if (tf >= t_end || tf + ITEMS <= t_out) continue;
        const int64_t oo = wi.out_off - D + tf;
        const bool all_in = (tf >= t_out) && (tf + ITEMS <= t_end);
        bool fast = false;
        if constexpr ((C::OUT == OUT_MORLET || C::OUT == OUT_CPLX) && sizeof(R) == 4)
          fast = all_in && ((reinterpret_cast<uintptr_t>(reinterpret_cast<V*>(P.out) + oo) & 15) == 0);
        if (fast) {
          // every position of the lane stored: pairs of outputs as 16-byte streaming stores
          float4* op = reinterpret_cast<float4*>(reinterpret_cast<V*>(P.out) + oo);
#pragma unroll
          for (int i = 0; i < ITEMS; i += 2) {
            const V o0 = one(i);
            const V o1 = one(i + 1);
            __stcs(op + i / 2, make_float4((float)o0.x, (float)o0.y, (float)o1.x, (float)o1.y));
          }
        } else {
          V prev{};
#pragma unroll
          for (int i = 0; i < ITEMS; ++i) {
            const V o = one(i);
            store_item<C>(P, oo, i, o, prev, false, tf + i >= t_out && tf + i < t_end);
            prev = o;
          }
        }
      }
    }
    w = w1;
    w1 = __shfl_sync(0xffffffffu, w2, 0);
  }
  // the warp's TMA stores complete before it exits (its staging tile is freed with the CTA)
  if (tma_pending && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace msft
