// Single-pass lane-chunk scan for short windows (compensated FP32, SFT, real input, Morlet output).
//
// The warp kernel's two passes and warp scan cost about as much as the recursion itself. When the
// window is short, each lane can instead own a contiguous chunk of C positions of a row and run the
// recursion through it once, from a zero state a prologue of >= 2L positions before the chunk
// (samples before chunk start - 2L count as zero, so the state is exact from the chunk's first
// position on: the window-segment restart of the warp kernel, per lane). The recursion is the SFT's
// 2L-sample form G <- rho G + (x[t] - x[t - 2L]), V = G + x[t - 2L] (see wscan_kernel.cuh), with the
// direct-method combine of Sec. III-A; FP32 throughout, its history bounded by prologue + C.
// Each step multiplies by rho = e^{-i theta} as three shears (x += t y; y -= s x; x += t y with
// t = tan(theta/2), s = sin(theta)): the same operation count as a complex multiply, but the map has
// determinant exactly one and its angle error is relative to theta, so the thousands of rotations a
// lane applies drift far less in magnitude and phase than repeated products with a rounded rho.
//
// The 32 chunks of a warp lie C positions apart, so every global access goes through this warp's
// shared buffers, transposed:
//  - inputs: per step of 16 positions the warp copies the 32 lanes' runs of x[t] and x[t - 2L] into
//    shared memory as 16-byte pieces (5 per run, covering a misalignment of up to 3 samples;
//    consecutive lanes take consecutive pieces) with cp.async into the step's buffer (two buffers,
//    alternating). The copies of step k + 1 are issued as soon as step k's runs are in registers,
//    so they overlap step k's arithmetic; each lane reads its run back from a padded 80-byte row
//    and shifts it by the run's misalignment, which is the same for every lane and step;
//  - outputs: a lane's 16 complex outputs of a step are 128 contiguous bytes, and the 32 lanes'
//    pieces lie one chunk (8 C bytes) apart. When every lane's outputs of the step are in range,
//    the lanes write them as the 32 rows of a 4 KB tile in the buffer just read (128-byte
//    swizzle), which leaves as one TMA tensor store through a map of the output buffer viewed as
//    rows of one chunk (one map per chunk length, up to four). The copies of step k + 2 into the
//    same buffer wait until the store has read it. Without a map, such steps use four 256-bit stores
//    of whole sectors per lane (the plan starts every row's chunks on an output element that is a
//    multiple of 4). Other steps (those that touch the ends of the row, or a misaligned output
//    buffer) go through a padded 144-byte row per lane and are stored as masked 16-byte pieces,
//    eight lanes per row.
// Every bank access is conflict-free (row strides of 20 and 36 words).
//
// Work item fields (see WorkItem): t_a = first position of lane 0's chunk, n_sub = C (multiple of
// 16), t_dom = prologue (multiple of 16, >= 2L), t_out = D and t_end = D + N bound the stored
// positions.
#pragma once

#include "scan_kernel.cuh"

namespace msft {

constexpr int LS_WARPS = 4;                  // warps per CTA (shared memory per warp: 10 KB)
constexpr int LS_ITEMS = 16;                 // positions per lane per step
constexpr int LS_PIECES = 5;                 // 16-byte input pieces per lane run (20 samples)
constexpr int LS_RUN_F4 = 32 * LS_PIECES;    // float4 per input run buffer of a warp (160)
constexpr int LS_BUF_F4 = 2 * LS_RUN_F4;     // one step's lead + lag buffers (320 float4 = 5120 B); the
                                             // output rows (32 x 9 float4 = 4608 B) reuse them
static_assert(32 * 9 <= LS_BUF_F4, "output rows fit in the input buffers");

// v[i] = row[r + i] for the uniform shift r in [0, 3]
__device__ __forceinline__ void ls_shift(const float (&row)[4 * LS_PIECES], int r, float (&v)[LS_ITEMS]) {
  if (r == 0) {
#pragma unroll
    for (int i = 0; i < LS_ITEMS; ++i) v[i] = row[i];
  } else if (r == 1) {
#pragma unroll
    for (int i = 0; i < LS_ITEMS; ++i) v[i] = row[i + 1];
  } else if (r == 2) {
#pragma unroll
    for (int i = 0; i < LS_ITEMS; ++i) v[i] = row[i + 2];
  } else {
#pragma unroll
    for (int i = 0; i < LS_ITEMS; ++i) v[i] = row[i + 3];
  }
}

// 16-byte asynchronous copy global -> shared; `bytes` = 16, or 0 to write zeros (nothing is read).
__device__ __forceinline__ void ls_cp16(float4* dst, const float* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void ls_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void ls_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Piece of samples [e, e + 4) of the n-sample buffer x into dst: asynchronous when inside the
// buffer, zeros when outside, element by element (synchronously) when it straddles an end.
__device__ __forceinline__ void ls_piece(float4* dst, const float* __restrict__ x, int64_t e, int64_t n) {
  if (e >= 0 && e + 4 <= n) {
    ls_cp16(dst, x + e, 16);
  } else if (e + 4 <= 0 || e >= n) {
    ls_cp16(dst, x, 0);
  } else {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (e + i >= 0 && e + i < n) v[i] = __ldg(x + e + i);
    *dst = make_float4(v[0], v[1], v[2], v[3]);
  }
}

__device__ __forceinline__ int64_t ls_floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int ls_clamp(int64_t v, int hi) { return (int)(v < 0 ? 0 : (v > hi ? hi : v)); }

template <class C>
__global__ void __launch_bounds__(LS_WARPS * 32, C::K <= 4 ? 4 : 2) lscan_kernel(const __grid_constant__ KParams P) {
  static_assert(std::is_same<typename C::R, float>::value && C::CH == 1 && C::OUT == OUT_MORLET && !C::ASFT,
                "the lane-chunk scan is built for the FP32 SFT Morlet transform");
  constexpr int K = C::K;
  const int lane = threadIdx.x & 31;
  // (1024-byte aligned buffers: a consumed input buffer doubles as a TMA staging tile)
  __shared__ __align__(1024) float4 s_buf[LS_WARPS][2][LS_BUF_F4];
  float4 (*const bufs)[LS_BUF_F4] = s_buf[threadIdx.x >> 5];
  const float* __restrict__ xg = reinterpret_cast<const float*>(P.x);
  const int64_t b0 = (int64_t)(reinterpret_cast<uintptr_t>(xg) >> 2);

  long long w = 0;
  if (lane == 0) w = (long long)atomicAdd(P.ticket, 1ull);
  w = __shfl_sync(0xffffffffu, w, 0);
  bool tma_pending = false;  // a TMA store may still be reading the buffer of the previous step
  while (w < P.n_work) {
    const WorkItem wi = P.work[w];
    long long w2 = 0;  // items are independent: claim the next one now
    if (lane == 0) w2 = (long long)atomicAdd(P.ticket, 1ull);

    const ScaleTab* tb = P.tabs + wi.scale;
    float2 sh[K];  // (tan(theta/2), sin(theta)) per term
    float cM[K], cL[K], cx = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      sh[j] = __ldg(&tb->f_shear[j]);
      cM[j] = tb->f_cM[j];
      cL[j] = tb->f_cL[j];
      cx += cM[j];
    }
    // positions relative to the row fit in 32 bits (the plan keeps rows below 2^30 positions)
    const int N = (int)wi.n, pro = (int)wi.t_dom, Cc = wi.n_sub, L2 = 2 * (int)tb->L;
    const int a0 = (int)wi.t_a - pro;             // lane 0's first processed position
    const int s_l = (int)wi.t_a + lane * Cc;      // this lane's first output position
    const int lo_l = s_l - L2 > 0 ? s_l - L2 : 0;  // samples before lo_l count as zero
    const int t_out = (int)wi.t_out, t_end = (int)wi.t_end;
    const float* __restrict__ xrow = xg + wi.x_off;
    // misalignment (in samples) of the lead and lagged runs, from their addresses; the same for
    // every lane and step since C and the step are multiples of 4 samples
    const int rl = (int)((b0 + wi.x_off + a0) & 3), rg = (int)((b0 + wi.x_off + a0 - L2) & 3);
    const int n_pro = pro / LS_ITEMS, n_steps = (pro + Cc) / LS_ITEMS;
    int off[LS_PIECES];  // this lane's input pieces: chunk c = pc / 5, piece q = pc % 5 -> c C + 4 q
#pragma unroll
    for (int r = 0; r < LS_PIECES; ++r) {
      const int pc = lane + 32 * r;
      off[r] = (pc / LS_PIECES) * Cc + 4 * (pc % LS_PIECES);
    }
    // the whole item reads inside the buffer (no per-piece bounds checks)
    const int64_t e0 = wi.x_off + a0;
    const int64_t span = 31LL * Cc + (int64_t)n_steps * LS_ITEMS + 4 * LS_PIECES;
    const bool inside = (e0 - L2 - 4 >= 0) && (e0 + span <= P.n_x);
    // Steps that need no input masks in any lane: the lead run needs lo_l <= p and p + 16 <= N, the
    // lagged run (output steps) lo_l <= p - 2L and p - 2L + 16 <= N, for p = p0 + 16 k.
    int kl_a, kh_a, kl_g, kh_g;
    {
      const int64_t p0 = a0 + (int64_t)lane * Cc;
      kl_a = ls_clamp(-ls_floordiv(p0 - lo_l, LS_ITEMS), n_steps);
      kh_a = ls_clamp(ls_floordiv(N - LS_ITEMS - p0, LS_ITEMS) + 1, n_steps);
      kl_g = ls_clamp(-ls_floordiv(p0 - lo_l - L2, LS_ITEMS), n_steps);
      kh_g = ls_clamp(ls_floordiv((int64_t)N + L2 - LS_ITEMS - p0, LS_ITEMS) + 1, n_steps);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        kl_a = max(kl_a, __shfl_xor_sync(0xffffffffu, kl_a, o));
        kh_a = min(kh_a, __shfl_xor_sync(0xffffffffu, kh_a, o));
        kl_g = max(kl_g, __shfl_xor_sync(0xffffffffu, kl_g, o));
        kh_g = min(kh_g, __shfl_xor_sync(0xffffffffu, kh_g, o));
      }
    }
    // 16-byte output pieces when the row's chunk starts are 16-byte aligned
    float2* const orow = reinterpret_cast<float2*>(P.out) + (wi.out_off - tb->D);
    const bool o16 = ((reinterpret_cast<uintptr_t>(orow + wi.t_a) & 15) == 0);
    const bool o32 = ((reinterpret_cast<uintptr_t>(orow + wi.t_a) & 31) == 0);
    const int so = (lane >> 3) * Cc + 2 * (lane & 7);  // this lane's store piece in round 0
    // TMA stores when the item's chunk length has a tensor map: (ys, rs) = view row and byte offset
    // in it of lane 0's outputs at the current output step; chunk c of the step lies c rows below
    int q = -1;
#pragma unroll
    for (int qq = 0; qq < 4; ++qq)
      if (P.lmap_c[qq] == Cc) q = qq;
    const int CB = 8 * Cc;
    int ys = 0, rs = 0;  // (view rows are below 2^31)
    if (q >= 0) {
      const int64_t A0 = 8LL * (wi.out_off - tb->D + wi.t_a);
      const int64_t y0 = ls_floordiv(A0, CB);
      ys = (int)y0;
      rs = (int)(A0 - y0 * CB);
    }

    // copies of step k into buffer k & 1
    auto issue = [&](int k) {
      float4* bl = bufs[k & 1];
      const int step0 = a0 + k * LS_ITEMS;
      const bool lag = k >= n_pro;  // the prologue reads no lagged samples
      if (inside) {
        const float* pl = xrow + (step0 - rl);
        const float* pg = xrow + (step0 - L2 - rg);
#pragma unroll
        for (int r = 0; r < LS_PIECES; ++r) {
          ls_cp16(bl + lane + 32 * r, pl + off[r], 16);
          if (lag) ls_cp16(bl + LS_RUN_F4 + lane + 32 * r, pg + off[r], 16);
        }
      } else {
        const int64_t el = wi.x_off + step0 - rl, eg = wi.x_off + step0 - L2 - rg;
#pragma unroll
        for (int r = 0; r < LS_PIECES; ++r) {
          ls_piece(bl + lane + 32 * r, xg, el + off[r], P.n_x);
          if (lag) ls_piece(bl + LS_RUN_F4 + lane + 32 * r, xg, eg + off[r], P.n_x);
        }
      }
      ls_commit();
    };

    float2 S[K];
#pragma unroll
    for (int j = 0; j < K; ++j) S[j] = make_float2(0.f, 0.f);

    // Buffer k & 1 takes the copies of step k; they are issued once step k - 1's inputs are in
    // registers, after the TMA store staged in that buffer two steps earlier has read it.
    if (tma_pending) {
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncwarp();
      tma_pending = false;
    }
    issue(0);
    for (int k = 0; k < n_steps; ++k) {
      ls_wait_all();
      __syncwarp();
      float4* bl = bufs[k & 1];
      const int step0 = a0 + k * LS_ITEMS;  // lane 0's first position of this step
      const bool pro_step = k < n_pro;                   // warp-uniform
      float xa[LS_ITEMS], xl[LS_ITEMS];
      {
        float row[4 * LS_PIECES];
#pragma unroll
        for (int q = 0; q < LS_PIECES; ++q) reinterpret_cast<float4*>(row)[q] = bl[lane * LS_PIECES + q];
        ls_shift(row, rl, xa);
        if (!pro_step) {
#pragma unroll
          for (int q = 0; q < LS_PIECES; ++q) reinterpret_cast<float4*>(row)[q] = bl[LS_RUN_F4 + lane * LS_PIECES + q];
          ls_shift(row, rg, xl);
        }
      }
      __syncwarp();
      if (k + 1 < n_steps) {
        if (tma_pending) {
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          __syncwarp();
          tma_pending = false;
        }
        issue(k + 1);
      }
      if (k < kl_a || k >= kh_a || (!pro_step && (k < kl_g || k >= kh_g))) {  // warp-uniform
        const int p = step0 + lane * Cc;
#pragma unroll
        for (int i = 0; i < LS_ITEMS; ++i) {
          const int t = p + i;
          if (t < lo_l || t >= N) xa[i] = 0.f;
          if (t - L2 < lo_l || t - L2 >= N) xl[i] = 0.f;
        }
      }
      if (pro_step) {  // x[t - 2L] is before lo_l throughout the prologue: the input is x[t] alone
#pragma unroll
        for (int i = 0; i < LS_ITEMS; ++i) {
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const float x1 = fmaf(sh[j].x, S[j].y, S[j].x);
            S[j].y = fmaf(-sh[j].y, x1, S[j].y);
            S[j].x = fmaf(sh[j].x, S[j].y, x1 + xa[i]);
          }
        }
        continue;
      }
      // ---- output step: recursion and combine ----
      auto one = [&](int i) -> float2 {
        const float d = xa[i] - xl[i];
        float ox = 0.f, oy = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const float x1 = fmaf(sh[j].x, S[j].y, S[j].x);
          S[j].y = fmaf(-sh[j].y, x1, S[j].y);
          S[j].x = fmaf(sh[j].x, S[j].y, x1 + d);
          ox = fmaf(cM[j], S[j].x, ox);
          oy = fmaf(cL[j], S[j].y, oy);
        }
        return make_float2(fmaf(cx, xl[i], ox), oy);
      };
      const bool full = step0 >= t_out && step0 + 31 * Cc + LS_ITEMS <= t_end;  // warp-uniform
      const int ys_k = ys, rs_k = rs;
      if (q >= 0) {  // the next output step's position in the view
        rs += 128;
        if (rs >= CB) {
          rs -= CB;
          ++ys;
        }
      }
      if (q >= 0 && full && rs_k + 128 <= CB && ys_k >= 0 && ys_k + 32 <= P.lmap_rows[q]) {
        // every lane's 16 outputs are in range and in one view row: the lanes' 128-byte rows are
        // staged in the buffer just read (128-byte swizzle) and leave as one TMA tensor store
#pragma unroll
        for (int i = 0; i < LS_ITEMS; i += 2) {
          const float2 o0 = one(i), o1 = one(i + 1);
          bl[lane * 8 + ((i / 2) ^ (lane & 7))] = make_float4(o0.x, o0.y, o1.x, o1.y);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                           reinterpret_cast<uint64_t>(&P.lmap[q])),
                       "r"(rs_k >> 2), "r"(ys_k), "r"((uint32_t)__cvta_generic_to_shared(bl))
                       : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        tma_pending = true;
        continue;
      }
      if (o32 && full) {
        // every lane's 16 outputs are in range: four 32-byte stores of whole sectors per lane
        float2* op = orow + (step0 + lane * Cc);
#pragma unroll
        for (int i = 0; i < LS_ITEMS; i += 4) {
          const float2 o0 = one(i), o1 = one(i + 1), o2 = one(i + 2), o3 = one(i + 3);
          asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(op + i),
                       "f"(o0.x), "f"(o0.y), "f"(o1.x), "f"(o1.y), "f"(o2.x), "f"(o2.y), "f"(o3.x), "f"(o3.y)
                       : "memory");
        }
        continue;
      }
#pragma unroll
      for (int i = 0; i < LS_ITEMS; i += 2) {
        const float2 o0 = one(i), o1 = one(i + 1);
        bl[lane * 9 + i / 2] = make_float4(o0.x, o0.y, o1.x, o1.y);
      }
      __syncwarp();
      // ---- cooperative stores: row c's 16-byte piece q holds positions p_c + 2q, p_c + 2q + 1 ----
      if (o16 && step0 >= t_out && step0 + 31 * Cc + LS_ITEMS <= t_end) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int pc = lane + 32 * r;
          __stcs(reinterpret_cast<float4*>(orow + (step0 + so + 4 * r * Cc)), bl[(pc >> 3) * 9 + (pc & 7)]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int pc = lane + 32 * r;
          const int pos = step0 + so + 4 * r * Cc;
          const bool in0 = pos >= t_out && pos < t_end;
          const bool in1 = pos + 1 >= t_out && pos + 1 < t_end;
          const float4 v = bl[(pc >> 3) * 9 + (pc & 7)];
          if (in0 && in1 && o16) {
            __stcs(reinterpret_cast<float4*>(orow + pos), v);
          } else {
            if (in0) __stcs(orow + pos, make_float2(v.x, v.y));
            if (in1) __stcs(orow + pos + 1, make_float2(v.z, v.w));
          }
        }
      }
      __syncwarp();
    }
    w = __shfl_sync(0xffffffffu, w2, 0);
  }
  // the warp's TMA stores complete before it exits (its buffers are freed with the CTA)
  if (tma_pending && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace msft
