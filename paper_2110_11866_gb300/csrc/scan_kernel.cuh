// The SFT / ASFT window-sum scan (Sec. II-B, II-D, III-A) as one persistent sm_103a kernel.
//
// For every harmonic p_j = p0 + j (beta = pi / L) and every scan position t the kernel keeps the
// window state of the 2L+1 samples x[t-2L .. t]. Two forms are built:
//
//  Kernel-integral form (FORM_KI), the paper's GPU formulation (eqs. kernel, kernelInter,
//  kernelIntZenka): modulate a[t] = x[t] e^{i beta p t}, scan the lagged difference
//  d[t] = a[t] - a[t-2L-1] (its prefix is the window sum u_(2L+1)[t]), then demodulate
//  e^{-i beta p t} u_(2L+1)[t] and combine. Phases are advanced by a fixed step from a per-tile
//  anchor that is computed in FP64 from the exact integer (p t) mod 2L.
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
// Work decomposition: a row (signal, scale) is cut into sub-tiles of T = THREADS * ITEMS positions
// on the output grid. A CTA takes work items from a global counter (so every predecessor of a
// claimed item is already running) and, per sub-tile:
//   1. loads x[t] and x[t - 2L - 1] for its ITEMS consecutive positions per thread,
//   2. pass 1: runs the recursion from a zero state -> per-thread aggregate,
//   3. warp-shuffle scan of the aggregates (rotation powers rho^{ITEMS 2^l}),
//   4. warp 0 combines the 8 warp totals, publishes the tile aggregate, looks back over the row's
//      earlier tiles (decoupled look-back, bounded waits) or takes the carry of its own previous
//      sub-tile, and publishes the inclusive state (carries in CR precision: FP64 for the
//      compensated form),
//   5. pass 2: reruns the recursion from each thread's exact start state and writes the outputs.
// Rows with short windows (2L+1 <= 2T) use no look-back at all: the work item starts 2L samples
// before its first output with a zero state, so no error accumulates along the row.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace msft {

enum { FORM_KI = 1, FORM_RF = 2 };
enum { OUT_MORLET = 0, OUT_REAL = 1, OUT_ADJ = 2 };

template <typename R_, typename CR_, int K_, int FORM_, int OUT_, bool ASFT_, int ITEMS_>
struct Cfg {
  using R = R_;
  using CR = CR_;
  using V = typename C2<R_>::T;
  using CV = typename C2<CR_>::T;
  static constexpr int K = K_;
  static constexpr int FORM = FORM_;
  static constexpr int OUT = OUT_;
  static constexpr bool ASFT = ASFT_;
  static constexpr int ITEMS = ITEMS_;
  static constexpr int CH = (OUT_ == OUT_ADJ) ? 2 : 1;
  static constexpr int NT = CH * K_;
  static constexpr int T = THREADS * ITEMS_;
  static_assert(FORM_ == FORM_RF || CH == 1, "kernel-integral form is built for real input only");
  static_assert(NT <= 32, "one lane per scanned value in the block phase");
};

template <class C>
struct Smem {
  using R = typename C::R;
  using V = typename C::V;
  using CV = typename C::CV;
  WorkItem wi;
  ChainDesc ch;
  long long work;
  int cur_scale;
  int64_t L, D;
  int32_t p0;
  // staged per scale
  V rho[C::K];
  V pw_thr[5][C::K];
  V pw_lane[32][C::K];
  V pw_wofs_r[8][C::K];
  R cM[C::K], cL[C::K];
  V E;
  R kappa;
  CV pw_warp_c[C::K];
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
// loads and stores
// ------------------------------------------------------------------------------------------------

// v[i] = p[t + i] if lo <= t + i < hi, else 0. 128-bit loads when the run is in range and aligned.
template <typename E, int N>
__device__ __forceinline__ void load_run(const E* __restrict__ p, int64_t t, int64_t lo, int64_t hi,
                                         E (&v)[N]) {
  if (t >= lo && t + N <= hi) {
    const E* q = p + t;
    constexpr int VEC = 16 / sizeof(E);
    if (VEC >= 1 && (reinterpret_cast<uintptr_t>(q) & 15) == 0) {
#pragma unroll
      for (int i = 0; i < N; i += (VEC > 0 ? VEC : 1)) {
        const int4 u = __ldg(reinterpret_cast<const int4*>(q + i));
        const E* e = reinterpret_cast<const E*>(&u);
#pragma unroll
        for (int j = 0; j < VEC; ++j) v[i + j] = e[j];
      }
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) v[i] = __ldg(q + i);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int64_t u = t + i;
      v[i] = (u >= lo && u < hi) ? __ldg(p + u) : E{};
    }
  }
}

__device__ __forceinline__ void st_cs(float2* p, float2 a, float2 b) {
  __stcs(reinterpret_cast<float4*>(p), make_float4(a.x, a.y, b.x, b.y));
}

// ------------------------------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------------------------------

template <class C>
__global__ void __launch_bounds__(THREADS) scan_kernel(const KParams P) {
  using R = typename C::R;
  using CR = typename C::CR;
  using V = typename C::V;
  using CV = typename C::CV;
  constexpr int K = C::K, NT = C::NT, CH = C::CH, ITEMS = C::ITEMS, T = C::T;
  constexpr bool ROT = (C::FORM == FORM_RF);
  // element type of one input sample (real, or complex for the adjoint's two channels)
  using EIn = typename std::conditional<CH == 2, V, R>::type;

  __shared__ Smem<C> s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s.cur_scale = -1;

  for (;;) {
    __syncthreads();  // everyone is done with the previous work item
    if (tid == 0) {
      const long long w = (long long)atomicAdd(P.ticket, 1ull);
      s.work = w;
      if (w < P.n_work) {
        s.wi = P.work[w];
        s.ch = P.chains[s.wi.chain];
      }
    }
    __syncthreads();
    if (s.work >= P.n_work) return;
    const WorkItem wi = s.wi;
    const ChainDesc ch = s.ch;

    if (ch.scale != s.cur_scale) {  // stage this scale's constants (uniform branch)
      const ScaleTab* tb = P.tabs + ch.scale;
      for (int i = tid; i < K; i += THREADS) {
        s.rho[i] = conv2<V>(tb->rho[i]);
        s.cM[i] = (R)tb->cM[i];
        s.cL[i] = (C::OUT == OUT_ADJ) ? (R)(-tb->cL[i]) : (R)tb->cL[i];
        s.pw_warp_c[i] = conv2<CV>(tb->pw_warp[i]);
      }
      for (int i = tid; i < 5 * K; i += THREADS) s.pw_thr[i / K][i % K] = conv2<V>(tb->pw_thr[i / K][i % K]);
      for (int i = tid; i < 32 * K; i += THREADS) s.pw_lane[i / K][i % K] = conv2<V>(tb->pw_lane[i / K][i % K]);
      for (int i = tid; i < 8 * K; i += THREADS) {
        s.pw_wofs_r[i / K][i % K] = conv2<V>(tb->pw_wofs[i / K][i % K]);
        s.pw_wofs_c[i / K][i % K] = conv2<CV>(tb->pw_wofs[i / K][i % K]);
      }
      for (int i = tid; i < 33 * K; i += THREADS) s.pw_tile_c[i / K][i % K] = conv2<CV>(tb->pw_tile[i / K][i % K]);
      if (tid == 0) {
        s.E = conv2<V>(tb->E);
        s.kappa = (R)tb->kappa;
        s.L = tb->L;
        s.D = tb->D;
        s.p0 = tb->p0;
      }
      __syncthreads();
      if (tid == 0) s.cur_scale = ch.scale;
    }
    const int64_t L = s.L, D = s.D, Wl = 2 * L + 1;
    const R kap = s.kappa;

    const EIn* __restrict__ xs = reinterpret_cast<const EIn*>(P.x) + ch.x_off;
    const int64_t N = ch.n;
    const int64_t lo = wi.t_dom;  // samples before t_dom count as zero (>= 0)
    if (tid < NT) s.carry[tid] = CV{};

    for (int sub = 0; sub < wi.n_sub; ++sub) {
      const int64_t k = wi.k_first + sub;
      const int64_t t0 = D + k * (int64_t)T;
      const int64_t tf = t0 + (int64_t)tid * ITEMS;  // this thread's first position
      const bool store = (k >= wi.k_out);

      if constexpr (!ROT) {
        // phase anchor e^{i beta p (t0 - 1)} from the exact integer (p (t0-1)) mod 2L, in FP64
        if (tid < K) {
          const long long p = s.p0 + tid, m = 2 * L;
          long long r = (p * (long long)(t0 - 1)) % m;
          if (r < 0) r += m;
          double sn, cs;
          sincospi((double)r / (double)L, &sn, &cs);
          s.base[tid] = cmake<R>((R)cs, (R)sn);
        }
        __syncthreads();
      }

      // ---- 1. loads ----
      EIn xa[ITEMS], xl[ITEMS];
      const bool live = (tf + ITEMS > lo && tf < N) || (tf - Wl + ITEMS > lo && tf - Wl < N);
      if (live) {
        load_run<EIn, ITEMS>(xs, tf, lo, N, xa);
        load_run<EIn, ITEMS>(xs, tf - Wl, lo, N, xl);
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
            else { B[v].x += u.x; B[v].y += u.y; }
          }
        }
      }
      if (lane == 31) {
#pragma unroll
        for (int v = 0; v < NT; ++v) s.wtot[warp][v] = B[v];
      }
      // exclusive value: the inclusive of the previous lane
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        V u = shfl_up2(B[v], 1);
        if (lane == 0) u = V{};
        B[v] = u;
      }
      __syncthreads();

      // ---- 4. block phase: warp 0 ----
      if (warp == 0) {
        // tile aggregate A (zero entering state)
        CV A = CV{};
        if (lane < NT) {
#pragma unroll
          for (int w = 0; w < WARPS; ++w) {
            const double2 t2 = wide2<V>(s.wtot[w][lane]);
            CV twc;
            twc.x = (CR)t2.x;
            twc.y = (CR)t2.y;
            if constexpr (ROT) A = cfma(s.pw_warp_c[lane % K], A, twc);
            else { A.x += twc.x; A.y += twc.y; }
          }
        }
        const bool lookback = (sub == 0) && (wi.slot >= 0);
        if (lookback) {
          const int64_t slot = wi.slot;
          CV* aggp = reinterpret_cast<CV*>(P.agg);
          CV* inclp = reinterpret_cast<CV*>(P.incl);
          if (slot == wi.slot_first) {
            if (lane < NT) s.carry[lane] = CV{};
          } else {
            // publish the aggregate, then look back
            if (lane < NT) {
              __stcg(aggp + slot * NT + lane, A);
              __threadfence();
            }
            __syncwarp();
            if (lane == 0) st_release(P.flags + slot, ST_AGG);
            if (lane < NT) {
              s.carry[lane] = CV{};
              s.rot[lane] = ROT ? conv2<CV>(make_double2(1.0, 0.0)) : CV{};
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
              // sum of predecessor values, lane q rotated by rho^{T q} (times rho^{32 T} per batch)
              for (int v = 0; v < NT; ++v) {
                CV val = CV{};
                if (lane <= first && valid && !forced) {
                  const CV* src = (f == ST_INCL) ? inclp : aggp;
                  val = ld_cg2<CV>(src + j * NT + v);
                  if constexpr (ROT) val = cmul(s.pw_tile_c[lane][v % K], val);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                  const CV u = shfl_xor2(val, o);
                  val.x += u.x;
                  val.y += u.y;
                }
                if (lane == 0) {
                  if constexpr (ROT) s.carry[v] = cfma(s.rot[v], val, s.carry[v]);
                  else { s.carry[v].x += val.x; s.carry[v].y += val.y; }
                }
              }
              __syncwarp();
              if (first < 32) break;
              base -= 32;
              if constexpr (ROT) {
                if (lane < NT) s.rot[lane] = cmul(s.rot[lane], s.pw_tile_c[32][lane % K]);
              }
              __syncwarp();
            }
          }
          __syncwarp();
          // publish the inclusive state after this tile
          if (lane < NT) {
            CV inc = s.carry[lane];
            if constexpr (ROT) inc = cfma(s.pw_tile_c[1][lane % K], inc, A);
            else { inc.x += A.x; inc.y += A.y; }
            __stcg(inclp + slot * NT + lane, inc);
            __threadfence();
          }
          __syncwarp();
          if (lane == 0) st_release(P.flags + slot, ST_INCL);
        }
        __syncwarp();
        // start state of each warp, and the carry into the next sub-tile
        if (lane < NT) {
          const CV c0 = s.carry[lane];
          CV X = CV{};
#pragma unroll
          for (int w = 0; w < WARPS; ++w) {
            CV xw;
            if constexpr (ROT) xw = cfma(s.pw_wofs_c[w][lane % K], c0, X);
            else { xw.x = X.x + c0.x; xw.y = X.y + c0.y; }
            s.xw[w][lane] = cmake<R>((R)xw.x, (R)xw.y);
            const double2 t2 = wide2<V>(s.wtot[w][lane]);
            CV twc;
            twc.x = (CR)t2.x;
            twc.y = (CR)t2.y;
            if constexpr (ROT) X = cfma(s.pw_warp_c[lane % K], X, twc);
            else { X.x += twc.x; X.y += twc.y; }
          }
          CV nxt;
          if constexpr (ROT) nxt = cfma(s.pw_tile_c[1][lane % K], c0, A);
          else { nxt.x = c0.x + A.x; nxt.y = c0.y + A.y; }
          s.carry[lane] = nxt;
        }
      }
      __syncthreads();

      // ---- 5. pass 2: outputs ----
      const int64_t nf = tf - D;  // first output index of this thread
      if (!store || nf >= N || nf + ITEMS <= 0) continue;
      V S[NT];
#pragma unroll
      for (int v = 0; v < NT; ++v) {
        if constexpr (ROT) S[v] = cfma(s.pw_lane[lane][v % K], s.xw[warp][v], B[v]);
        else { S[v].x = s.xw[warp][v].x + B[v].x; S[v].y = s.xw[warp][v].y + B[v].y; }
      }
      V ph[ROT ? 1 : K];
      if constexpr (!ROT) {
#pragma unroll
        for (int j = 0; j < K; ++j) ph[j] = ph0[j];
      }
      const int64_t oo = ch.out_off + nf;
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        V o = V{};
        if constexpr (ROT) {
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
            const R qx = fma(pn.x, S[j].x, pn.y * S[j].y);   // conj(phase) * window sum
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
        // store output n = nf + i
        const int64_t n = nf + i;
        if constexpr (C::OUT == OUT_MORLET) {
          V* op = reinterpret_cast<V*>(P.out);
          if (n >= 0 && n < N) {
            if constexpr (sizeof(R) == 4) __stcs(reinterpret_cast<float2*>(op + (oo + i)), reinterpret_cast<const float2&>(o));
            else __stcs(reinterpret_cast<double2*>(op + (oo + i)), reinterpret_cast<const double2&>(o));
          }
        } else if constexpr (C::OUT == OUT_ADJ) {
          R* op = reinterpret_cast<R*>(P.out);
          if (n >= 0 && n < N) op[oo + i] = P.accumulate ? op[oo + i] + o.x : o.x;
        } else {
          R* op = reinterpret_cast<R*>(P.out);
          if (n >= 0 && n < N) __stcs(op + (oo + i), o.x);
        }
      }
    }
  }
}

}  // namespace msft
