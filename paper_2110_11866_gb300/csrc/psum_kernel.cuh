// Lag-free prefix sums of the rotating-form recursion at tile ends: the start states of the warp
// kernel's long-window rows (compensated FP32, SFT, real input).
//
// For one row and one harmonic let P(t) = sum_{0 <= u <= t} rho^{t-u} x[u], so P(t) = rho P(t-1) + x[t].
// Substituting into the rotating form V[t] = rho V[t-1] + x[t] - kappa rho x[t-2L-1] shows that
//     V(t) = P(t) - kappa rho P(t - 2L - 1)
// (both sides obey the same recursion and vanish for t < 0). P is the running sum behind the
// sliding sum of Sec. II-B without its lagged subtraction; with |rho| = 1 it grows without bound
// when x holds the harmonic's own frequency, so it is kept in two-float precision. A window state
// taken as the difference of two such values then carries only the FP32 rounding of the tile sums
// inside its own window: a work item of the warp kernel can start anywhere in a row from an exact
// state, with neither a look-back nor a 2L-sample prologue.
//
// Tiles are 512 positions (32 lanes x 16 samples), tile 0 of a row starting at the position t_grid
// whose input element is 32-byte aligned. A work item is a chunk of up to 8 tiles (4096 positions,
// the unit of the pw_tile powers) of one row, taken by one warp:
//   per tile: lane-serial Horner sum of its 16 samples, a warp reduction weighted by
//             rho^{16 (31 - lane)} -> the tile sum G (FP32), and the chunk aggregate in FP32;
//   warp-level decoupled look-back over the row's earlier chunks (two-float) -> P before the chunk;
//   P at the end of every tile of the chunk, two-float, stored for the warp kernel.
#pragma once

#include "scan_kernel.cuh"

namespace msft {

constexpr int PS_TILE = 512;                // positions per tile of the prefix sums
constexpr int PS_CHUNK = 8;                 // tiles per prefix-sum work item
static_assert(PS_TILE * PS_CHUNK == THREADS * 16, "a chunk is one pw_tile unit");

// Two-float complex from the hi / lo FP32 copies of rho^{512} of term j.
__device__ __forceinline__ DFC dfc_rho512(const ScaleTab* tb, int j) {
  const float2 h = __ldg(&tb->f_pwt[0][j]);
  const float2 l = __ldg(&tb->f_pwt[1][j]);
  return DFC{DF{h.x, l.x}, DF{h.y, l.y}};
}

// Lane 0 stores the NT values held by lanes 0 .. NT-1 and then releases the status flag, so the
// values are visible at GPU scope before the flag (one thread, program order + release; no fence).
template <int NT>
__device__ __forceinline__ void publish(DFC* dst, uint32_t* flag, uint32_t status, DFC mine, int lane) {
#pragma unroll
  for (int v = 0; v < NT; ++v) {
    const DFC val = CarryOps<DFC>::shfl_idx(mine, v);
    if (lane == 0) st_cg2(dst + v, val);
  }
  if (lane == 0) st_release(flag, status);
}

// Warp-level decoupled look-back in two-float precision. Lane v < NT holds `mine`, the aggregate of
// term v over this item; the function publishes it (unless the item is the first of its chain),
// sums the predecessors' published values back to the first inclusive one, each rotated by
// rho^{4096 d} for a predecessor ending 4096 d positions before this item, and returns in lane v
// the state entering the item. Every wait is bounded by P.spin_limit polls; on timeout the error
// word is set and unpublished predecessors count as zero.
template <int NT>
__device__ __forceinline__ DFC warp_lookback(const KParams& P, int64_t slot, int64_t slot_first, DFC mine,
                                             const ScaleTab* tb, int lane) {
  using CO = CarryOps<DFC>;
  DFC carry = CO::zero();
  if (slot == slot_first) return carry;
  DFC* aggp = reinterpret_cast<DFC*>(P.agg);
  const DFC* inclp = reinterpret_cast<const DFC*>(P.incl);
  publish<NT>(aggp + slot * NT, P.flags + slot, ST_AGG, mine, lane);
  DFC rot = CO::one();
  int64_t base = slot - 1;
  long long polls = 0;
  bool timed_out = false;
  for (;;) {
    const int64_t j = base - lane;
    const bool valid = (j >= slot_first);
    uint32_t f = ST_INCL;
    bool forced = false;
    unsigned incl_mask;
    for (;;) {
      f = valid ? ld_acquire(P.flags + j) : ST_INCL;
      forced = timed_out && f == 0;
      if (forced) f = ST_INCL;
      incl_mask = __ballot_sync(0xffffffffu, f == ST_INCL);
      const unsigned zero_mask = __ballot_sync(0xffffffffu, f == 0);
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
    // lanes 0 .. first contribute: a butterfly over the smallest power of two covering them
    int span = 1;
    while (span < first + 1 && span < 32) span <<= 1;
#pragma unroll
    for (int v = 0; v < NT; ++v) {
      DFC val = CO::zero();
      if (use) {
        const DFC* src = (f == ST_INCL) ? inclp : aggp;
        val = ld_cg2<DFC>(src + j * NT + v);
        if (lane > 0) val = CO::mul(dfc_from_f4(__ldg(&tb->c_pw_tile[lane][v])), val);
      }
      for (int o = span >> 1; o > 0; o >>= 1) val = CO::add(val, CO::shfl_xor(val, o));
      val = CO::shfl_idx(val, 0);
      if (lane == v) carry = CO::add(CO::mul(rot, val), carry);
    }
    if (first < 32) break;
    base -= 32;
    if (lane < NT) rot = CO::mul(rot, dfc_from_f4(__ldg(&tb->c_pw_tile[32][lane])));
  }
  return carry;
}

// Sum of 16 samples with the lane's weight: returns w sum_i rho^{15 - i} x_i for rho = e^{-i theta}.
// The sum runs as the real second-order recurrence s_i = x_i + 2 cos(theta) s_{i-1} - s_{i-2} in
// Reinsch's form, which stays accurate for small theta: with lam = 4 sin^2(theta / 2),
//     d_i = d_{i-1} + x_i - lam s_{i-1},  s_i = s_{i-1} + d_i,
// and at the end sum_i rho^{15-i} x_i = (d_15 + (lam / 2) s_14) - i sin(theta) s_14 with
// s_14 = s_15 - d_15. Three operations per sample and term instead of a complex rotation's five,
// issued for two terms at a time (packed FP32).
template <int K, int ITEMS>
__device__ __forceinline__ void lane_sums(const float (&xa)[ITEMS], const float2 (&rho)[K], const float (&lam)[K],
                                          const float2 (&w)[K], float2 (&b)[K]) {
  float s[K], d[K];
  reinsch_pk<K, ITEMS>(xa, lam, d, s);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float s14 = s[j] - d[j];
    b[j] = cmul(make_float2(fmaf(0.5f * lam[j], s14, d[j]), rho[j].y * s14), w[j]);
  }
}

// The same weighted lane sum w sum_i rho^{15 - i} x_i for any rho (the damped rho of the ASFT, the
// non-harmonic rho of the multiplication method), by Horner's rule b <- rho b + x_i from zero: four
// operations per sample and term pair, two terms per instruction.
template <int K, int ITEMS>
__device__ __forceinline__ void lane_sums_horner(const float (&xa)[ITEMS], const float2 (&rho)[K],
                                                 const float2 (&w)[K], float2 (&b)[K]) {
  constexpr int H = Pairs<K>::H;
  float2 rx2[H], ry2[H], nry2[H], X2[H], Y2[H];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    const bool two = 2 * h + 1 < K;
    const float2 r0 = rho[2 * h], r1 = two ? rho[2 * h + 1] : make_float2(0.f, 0.f);
    rx2[h] = make_float2(r0.x, r1.x);
    ry2[h] = make_float2(r0.y, r1.y);
    nry2[h] = make_float2(-r0.y, -r1.y);
    X2[h] = Y2[h] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const float2 xv2 = pk_dup(xa[i]);
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float2 vr = pk_fma(rx2[h], X2[h], pk_fma(nry2[h], Y2[h], xv2));
      Y2[h] = pk_fma(ry2[h], X2[h], pk_mul(rx2[h], Y2[h]));
      X2[h] = vr;
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float2 v = (j & 1) ? make_float2(X2[j >> 1].y, Y2[j >> 1].y) : make_float2(X2[j >> 1].x, Y2[j >> 1].x);
    b[j] = cmul(v, w[j]);
  }
}

// Sum over the warp of each b[j] (all lanes receive the sums); returns the sum of term `lane`
// (zero in lanes >= K).
template <int K>
__device__ __forceinline__ float2 warp_tile_sum(float2 (&b)[K], int lane) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float2 u = shfl_xor2(b[j], o);
      b[j].x += u.x;
      b[j].y += u.y;
    }
  }
  float2 g = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < K; ++j)
    if (lane == j) g = b[j];
  return g;
}

// Term count padded to a power of two, and lanes per term after a reduce-scatter.
template <int K> struct KPad {
  static constexpr int V = K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : 16;
  static constexpr int G = 32 / V;
};

// Reduce-scatter of b[0..K) (zero-padded to KP terms) over the warp: each butterfly level sends
// half of the lane's remaining terms to its partner and keeps the other half, so that after log2 KP
// levels a lane holds one term; the remaining levels complete that term's sum. Returns in every lane
// the warp sum of term lane / G (G = 32 / KP lanes per term; terms >= K are zero padding).
template <int K>
__device__ __forceinline__ float2 warp_sum_scatter(const float2 (&b)[K], int lane) {
  constexpr int KP = KPad<K>::V, G = KPad<K>::G;
  float2 cur[KP];
#pragma unroll
  for (int j = 0; j < KP; ++j) cur[j] = j < K ? b[j] : make_float2(0.f, 0.f);
  constexpr int LG = KP == 2 ? 1 : KP == 4 ? 2 : KP == 8 ? 3 : 4;  // log2 KP
#pragma unroll
  for (int lvl = 0; lvl < LG; ++lvl) {
    const int H = KP >> (lvl + 1), o = 16 >> lvl;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const float2 snd = up ? cur[h] : cur[h + H];
      const float2 kp = up ? cur[h + H] : cur[h];
      const float2 rcv = shfl_xor2(snd, o);
      cur[h] = make_float2(kp.x + rcv.x, kp.y + rcv.y);
    }
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const float2 u = shfl_xor2(cur[0], o);
    cur[0].x += u.x;
    cur[0].y += u.y;
  }
  return cur[0];
}

// State entering a start-state work item of the warp kernel, returned in Cw[j] (uniform across the
// warp, FP32). The warp kernel runs the SFT in its G form, G(t) = sum_{u = t-2L+1}^{t} rho^{t-u} x[u]
// = P(t) - rho^{2L} P(t - 2L) = P(t) - P(t - 2L). With b = wi.t_a a tile start and q = b - 1 - 2L:
//     G(b - 1) = P(b - 1) - P(q),
//     P(q)     = rho^{-(e - q)} (rho^{512} P(e - 512) + sum_{u = e-511}^{q} rho^{e-u} x[u])
// for the tile [e - 511, e] holding q; P at tile ends comes from the prefix sums, the partial tile
// sum from the samples. rho^{-(e-q)} = rho^{-16 a} rho^{-b} (e - q = 16 a + b) comes from two
// two-float tables, each entry rounded once from FP64 at the exact integer angle (|rho| = 1).
template <int K, int ITEMS>
__device__ __forceinline__ void start_state(const KParams& P, const WorkItem& wi, const ScaleTab* tb,
                                            const float2 (&rho)[K], int lane, float2 (&Cw)[K]) {
  using CO = CarryOps<DFC>;
  const int jl = lane < K ? lane : 0;
  const DFC* pb = reinterpret_cast<const DFC*>(P.pbuf) + wi.p_row * K;
  const int64_t L = tb->L;
  const int64_t kb = (wi.t_a - wi.t_grid) / PS_TILE;
  DFC v = CO::zero();
  if (kb >= 1) v = dfc_from_f4(__ldg(reinterpret_cast<const float4*>(pb + (kb - 1) * K + jl)));
  const int64_t q = wi.t_a - 1 - 2 * L;
  if (q >= 0) {  // warp-uniform
    const int64_t k0 = (q - wi.t_grid) / PS_TILE;
    const int64_t a0 = wi.t_grid + k0 * PS_TILE;
    const int m = (int)(a0 + PS_TILE - 1 - q);  // e - q, 0 .. 511
    const float* __restrict__ xs = reinterpret_cast<const float*>(P.x) + wi.x_off;
    float xa[ITEMS];
    load_run_v8<ITEMS>(xs, a0 + (int64_t)lane * ITEMS, 0, wi.n < q + 1 ? wi.n : q + 1, xa, P.n_x - wi.x_off);
    float2 wl[K], b[K];
    float lam[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      wl[j] = __ldg(&tb->f_pw_lane_t[j][31 - lane]);
      lam[j] = __ldg(&tb->f_lam[j]);
    }
    lane_sums<K, ITEMS>(xa, rho, lam, wl, b);
    DFC pt = CO::from(warp_tile_sum<K>(b, lane));
    if (k0 >= 1)
      pt = dfc_add(dfc_mul(dfc_rho512(tb, jl), dfc_from_f4(__ldg(reinterpret_cast<const float4*>(pb + (k0 - 1) * K + jl)))), pt);
    const DFC wm = dfc_mul(dfc_from_f4(__ldg(&tb->c_neg16[m >> 4][jl])), dfc_from_f4(__ldg(&tb->c_neg1[m & 15][jl])));
    v = dfc_add(v, dfc_neg(dfc_mul(wm, pt)));
  }
  const float2 vn = CO::narrow(v);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    Cw[j].x = __shfl_sync(0xffffffffu, vn.x, j);
    Cw[j].y = __shfl_sync(0xffffffffu, vn.y, j);
  }
}

// State entering a start-state item from a window sum of stored tile sums (used when the window
// spans few tiles compared with the item): with b = wi.t_a a tile start and u0 the window's first
// sample (b - 2L for the SFT's 2L-sample G form, b - 1 - 2L for the 2L + 1 samples of the damped
// form, HORNER),
//     G(b - 1) = sum_{k = k0}^{kb - 1} rho^{512 (kb - 1 - k)} G_k,
// G_k the FP32 tile sums sum_{u in tile k} rho^{e_k - u} x[u] (tsum_kernel), except that the tile
// k0 holding u0 contributes only its samples from u0 on (a masked tile sum computed here). The lanes
// of a term's group take the window's tiles in turn with FP32 running powers of rho^{512} (damped
// for the ASFT, so every partial product stays below one in magnitude).
template <int K, int ITEMS, bool HORNER = false>
__device__ __forceinline__ void start_state_window(const KParams& P, const WorkItem& wi, const ScaleTab* tb,
                                                   const float2 (&rho)[K], int lane, float2 (&Cw)[K]) {
  constexpr int G = KPad<K>::G;
  const int tl = lane / G, sl = lane % G, tq = tl < K ? tl : 0;
  const int64_t L = tb->L;
  const int64_t kb = (wi.t_a - wi.t_grid) / PS_TILE;
  const int64_t u0 = wi.t_a - 2 * L - (HORNER ? 1 : 0);
  int64_t k0 = 0;
  float2 gp = make_float2(0.f, 0.f);  // masked sum of tile k0 for this lane's term
  bool partial = false;
  if (u0 > wi.t_grid) {  // warp-uniform
    k0 = (u0 - wi.t_grid) / PS_TILE;
    const int64_t a0 = wi.t_grid + k0 * PS_TILE;
    if (u0 > a0) {
      partial = true;
      const float* __restrict__ xs = reinterpret_cast<const float*>(P.x) + wi.x_off;
      float xa[ITEMS];
      load_run_v8<ITEMS>(xs, a0 + (int64_t)lane * ITEMS, u0 > 0 ? u0 : 0, wi.n, xa, P.n_x - wi.x_off);
      float2 wl[K], b[K];
#pragma unroll
      for (int j = 0; j < K; ++j) wl[j] = __ldg(&tb->f_pw_lane_t[j][31 - lane]);
      if constexpr (HORNER) {
        lane_sums_horner<K, ITEMS>(xa, rho, wl, b);
      } else {
        float lam[K];
#pragma unroll
        for (int j = 0; j < K; ++j) lam[j] = __ldg(&tb->f_lam[j]);
        lane_sums<K, ITEMS>(xa, rho, lam, wl, b);
      }
      gp = warp_sum_scatter<K>(b, lane);
    }
  }
  const float2* gb = reinterpret_cast<const float2*>(P.pbuf) + wi.p_row * K;
  const float2 step = __ldg(&tb->f_pw512[G][tq]);  // rho^{512 G}
  float2 w = __ldg(&tb->f_pw512[sl][tq]);           // rho^{512 m} for m = sl
  float2 acc = make_float2(0.f, 0.f);
  const int64_t n_t = kb - k0;  // tiles k0 .. kb - 1
  for (int64_t m0 = 0; m0 < n_t; m0 += G) {
    const int64_t m = m0 + sl, k = kb - 1 - m;
    if (m < n_t && tl < K) {
      const float2 v = (partial && k == k0) ? gp : gb[k * K + tl];
      acc = cfma(w, v, acc);
    }
    w = cmul(w, step);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    Cw[j].x = __shfl_sync(0xffffffffu, acc.x, j * G);
    Cw[j].y = __shfl_sync(0xffffffffu, acc.y, j * G);
  }
}

constexpr bool TS_PF = true;  // a tile-sum chunk prefetched into L2 when claimed

// Tile sums only: G_k = sum_{u in tile k} rho^{e_k - u} x[u] for the tiles of a chunk, FP32, stored
// for start_state_window. No look-back, no prefix: chunks are independent. Lane sums by Reinsch's
// recurrence for the SFT's harmonics (|rho| = 1), by Horner's rule for the damped or non-harmonic
// rho of the ASFT and the multiplication method (C::ASFT).
template <class C>
__global__ void __launch_bounds__(THREADS, C::K <= 4 ? 4 : 2) tsum_kernel(const KParams P) {
  static_assert(std::is_same<typename C::R, float>::value && C::CH == 1 && C::ITEMS == 16,
                "tile sums are built for the FP32 real-input kernels");
  constexpr int K = C::K, ITEMS = C::ITEMS;
  constexpr int G = KPad<K>::G;
  const int lane = threadIdx.x & 31;
  const int tl = lane / G, sl = lane % G;

  long long w = 0;
  if (lane == 0) w = (long long)atomicAdd(P.ticket, 1ull);
  w = __shfl_sync(0xffffffffu, w, 0);
  while (w < P.n_work) {
    const WorkItem wi = P.work[w];
    long long w2 = 0;  // chunks are independent: claim the next one now
    if (lane == 0) w2 = (long long)atomicAdd(P.ticket, 1ull);
    const ScaleTab* tb = P.tabs + wi.scale;
    float2 rho[K], wl[K];
    float lam[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      rho[j] = tb->f_rho[j];
      wl[j] = __ldg(&tb->f_pw_lane_t[j][31 - lane]);
      lam[j] = __ldg(&tb->f_lam[j]);
    }
    const float* __restrict__ xs = reinterpret_cast<const float*>(P.x) + wi.x_off;
    const int64_t N = wi.n;
    float2* gb = reinterpret_cast<float2*>(P.pbuf) + wi.p_row * K;
    if (TS_PF && lane == 0) prefetch_l2(xs, N, wi.t_a, wi.t_a + (int64_t)wi.n_sub * PS_TILE);
#pragma unroll 1
    for (int k = 0; k < wi.n_sub; ++k) {
      const int64_t t0 = wi.t_a + (int64_t)k * PS_TILE;
      float2 g = make_float2(0.f, 0.f);
      if (t0 < N && t0 + PS_TILE > 0) {  // warp-uniform
        float xa[ITEMS];
        load_run_v8<ITEMS>(xs, t0 + (int64_t)lane * ITEMS, 0, N, xa, P.n_x - wi.x_off);
        float2 b[K];
        if constexpr (C::ASFT) lane_sums_horner<K, ITEMS>(xa, rho, wl, b);
        else lane_sums<K, ITEMS>(xa, rho, lam, wl, b);
        g = warp_sum_scatter<K>(b, lane);
      }
      if (sl == 0 && tl < K) gb[(int64_t)k * K + tl] = g;
    }
    w = __shfl_sync(0xffffffffu, w2, 0);
  }
}

template <class C>
__global__ void __launch_bounds__(THREADS, C::K <= 4 ? 3 : 2) psum_kernel(const KParams P) {
  static_assert(std::is_same<typename C::R, float>::value && C::CH == 1 && C::ITEMS == 16,
                "prefix sums are built for the FP32 real-input kernels");
  constexpr int K = C::K, ITEMS = C::ITEMS;
  constexpr int G = KPad<K>::G;                         // lanes per term after the reduce-scatter
  constexpr int OWN = G < PS_CHUNK ? G : PS_CHUNK;      // lanes of a term that own tiles
  constexpr int TPL = PS_CHUNK / OWN;                   // consecutive tiles per owner lane
  const int lane = threadIdx.x & 31;
  const int tl = lane / G;                 // this lane's term (>= K: padding)
  const int sl = lane % G;                 // slot in the term's lane group
  const int tq = tl < K ? tl : 0;          // table index
  const bool owner = tl < K && sl < OWN;   // owns tiles sl * TPL .. sl * TPL + TPL - 1

  long long w = 0;
  if (lane == 0) w = (long long)atomicAdd(P.ticket, 1ull);
  w = __shfl_sync(0xffffffffu, w, 0);
  while (w < P.n_work) {
    const WorkItem wi = P.work[w];
    const ScaleTab* tb = P.tabs + wi.scale;
    float2 rho[K], wl[K];
    float lam[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      rho[j] = tb->f_rho[j];
      wl[j] = __ldg(&tb->f_pw_lane_t[j][31 - lane]);  // rho^{16 (31 - lane)}
      lam[j] = __ldg(&tb->f_lam[j]);
    }
    const float* __restrict__ xs = reinterpret_cast<const float*>(P.x) + wi.x_off;
    const int64_t N = wi.n;
    const int n_sub = wi.n_sub;

    // tile sums G_k, kept by the owner lane of tile k for this lane's term
    float2 Gm[TPL];
#pragma unroll
    for (int r = 0; r < TPL; ++r) Gm[r] = make_float2(0.f, 0.f);
    if (lane == 0) prefetch_l2(xs, N, wi.t_a, wi.t_a + (int64_t)n_sub * PS_TILE);  // the chunk, into L2
    // (not unrolled: the unrolled chunk overflowed the instruction cache)
#pragma unroll 1
    for (int k = 0; k < PS_CHUNK; ++k) {
      const int64_t t0 = wi.t_a + (int64_t)k * PS_TILE;
      if (k < n_sub && t0 < N && t0 + PS_TILE > 0) {  // warp-uniform
        float xa[ITEMS];
        load_run_v8<ITEMS>(xs, t0 + (int64_t)lane * ITEMS, 0, N, xa, P.n_x - wi.x_off);
        float2 b[K];
        lane_sums<K, ITEMS>(xa, rho, lam, wl, b);
        const float2 g = warp_sum_scatter<K>(b, lane);
#pragma unroll
        for (int r = 0; r < TPL; ++r)
          if (sl * TPL + r == k) Gm[r] = g;
      }
    }
    // in-chunk prefix at each tile end (FP32): owner-local over its tiles, then a scan over the
    // owner slots of the term's lane group
    auto f32 = [&](int mm) {  // rho^{512 (mm + 1)} of this lane's term, FP32
      const float4 c = __ldg(&tb->c_pw_chunk[mm][tq]);
      return make_float2(c.x, c.z);
    };
    float2 loc[TPL];
    loc[0] = Gm[0];
#pragma unroll
    for (int r = 1; r < TPL; ++r) loc[r] = cfma(f32(0), loc[r - 1], Gm[r]);
    float2 inc = loc[TPL - 1];
#pragma unroll
    for (int o = 1; o < OWN; o <<= 1) {
      const float2 u = shfl_up2(inc, o);
      if (sl >= o) inc = cfma(f32(TPL * o - 1), u, inc);
    }
    float2 e = shfl_up2(inc, 1);
    if (sl == 0) e = make_float2(0.f, 0.f);
    float2 pre[TPL];
#pragma unroll
    for (int r = 0; r < TPL; ++r) pre[r] = cfma(f32(r), e, loc[r]);
    // chunk aggregate of term v into lane v, for the look-back
    const int k_last = n_sub - 1;
    float2 pl_last = pre[0];
#pragma unroll
    for (int r = 1; r < TPL; ++r)
      if (k_last % TPL == r) pl_last = pre[r];
    const int src = (lane < K ? lane : 0) * G + k_last / TPL;
    const float2 acc = make_float2(__shfl_sync(0xffffffffu, pl_last.x, src), __shfl_sync(0xffffffffu, pl_last.y, src));
    const DFC carry = warp_lookback<K>(P, wi.slot, wi.slot_first, CarryOps<DFC>::from(acc), tb, lane);
    // inclusive state after a full chunk, published at once for the successors' look-back
    if (n_sub == PS_CHUNK) {
      const DFC inc2 = dfc_add(dfc_mul(dfc_from_f4(__ldg(&tb->c_pw_tile[1][lane < K ? lane : 0])), carry),
                               CarryOps<DFC>::from(acc));
      publish<K>(reinterpret_cast<DFC*>(P.incl) + wi.slot * K, P.flags + wi.slot, ST_INCL, inc2, lane);
    }
    // P at the end of each owned tile: rho^{512 (k + 1)} carry + in-chunk prefix, two-float
    const DFC cy = CarryOps<DFC>::shfl_idx(carry, tq);
    DFC* pb = reinterpret_cast<DFC*>(P.pbuf) + wi.p_row * K;
    if (owner) {
#pragma unroll
      for (int r = 0; r < TPL; ++r) {
        const int k = sl * TPL + r;
        if (k < n_sub) {
          const DFC pk = dfc_add(dfc_mul(dfc_from_f4(__ldg(&tb->c_pw_chunk[k][tq])), cy), CarryOps<DFC>::from(pre[r]));
          st_cg2(pb + (int64_t)k * K + tl, pk);
        }
      }
    }
    if (lane == 0) w = (long long)atomicAdd(P.ticket, 1ull);
    w = __shfl_sync(0xffffffffu, w, 0);
  }
}

}  // namespace msft
