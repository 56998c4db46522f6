// How one (signal, scale) row is cut into work items. Shared by the plan (host) and the
// allocation-free entry point (host and device), so both decompose a row identically.
#pragma once

#include "common.cuh"

namespace msft {

constexpr int ITEMS_DEFAULT = 16;
constexpr long long TILE_DEFAULT = (long long)THREADS * ITEMS_DEFAULT;

// Segment policies.
//   SEG_RESTART: compensated FP32 SFT and the multiplication method. FP32 rounding leaves about one
//     unit of roundoff of |x| per sample in the carried window state and, with |rho| = 1, nothing
//     ever forgets it; restarting the scan from a zero state 2L samples before each segment bounds
//     that history to (segment + 2L) samples. Windows of 2L <= 2T samples: independent window
//     segments (a prologue of at most about a fifth of the segment). Longer windows: a look-back
//     chain per segment of max(4T, 4L) outputs.
//   SEG_ROW: FP64, and the damped ASFT in either FP32 precision (|rho| < 1 forgets the rounding
//     history). Windows of 2L <= 2T go to window segments as above (a segment restarted from a
//     zero state 2L samples before its first output is exact, since the window sum depends only on
//     the last 2L + 1 samples); longer windows keep one look-back chain per row.
//   SEG_PLAIN: plain FP32 SFT (whose error grows with the row length) and MORLET_FLAG_NO_HALO: one
//     look-back chain per row.
enum { SEG_RESTART = 0, SEG_ROW = 1, SEG_PLAIN = 2 };

struct RowSpec {
  long long N, L, D;   // row length, half window, output shift
  long long x_off;     // first input element of the row
  long long out_off;   // first output element of the row
  int scale;
  int align;           // input elements per 32 bytes (segment starts are aligned to it)
  int policy;
  int chain;           // row index stored in the work items
  long long wt;        // positions per step of a window segment: a CTA sub-tile, or one warp-tile
  int warp_window;     // 1: window segments go to the warp-independent kernel
  long long o_lo = 0, o_hi = 0;  // stored output positions [o_lo, o_hi); o_hi = 0: [D, D + N)
  int seg_mult = 16;   // warp windows: a segment runs about seg_mult * L positions (8, 12 or 16)
};

// The row description both the plan and the allocation-free entry point use: segment starts aligned
// to 32 bytes of input (elem_bytes per sample); window segments on the warp-independent kernel step
// by one warp-tile of 32 x 16 positions, on the CTA kernel by a tile of T positions.
__host__ __device__ inline RowSpec make_row_spec(long long N, long long L, long long D, long long x_off,
                                                 long long out_off, int scale, int elem_bytes, int policy,
                                                 int chain, bool warp_window, long long T, long long o_lo,
                                                 long long o_hi, int seg_mult) {
  RowSpec r{N, L, D, x_off, out_off, scale, 32 / elem_bytes, policy, chain,
            warp_window ? 32LL * ITEMS_DEFAULT : T, warp_window ? 1 : 0, o_lo, o_hi};
  r.seg_mult = seg_mult;
  return r;
}

__host__ __device__ inline long long ws_floordiv(long long a, long long b) {
  return (a >= 0) ? a / b : -((-a + b - 1) / b);
}

// Start-state items of a row whose tile k covers positions [t_grid + tile k, t_grid + tile (k + 1)):
// the tiles whose sums an item starting on tile kb reads (start_state_window). Its window begins at
// u0 = t_a - 2L (t_a - 2L - 1 for the Horner form's 2L + 1 samples), t_a = t_grid + tile kb; the
// tile holding u0 is summed by the item itself when u0 lies inside it (a masked sum), and positions
// before t_grid are zero, so the item reads the sums of the tiles [a, b) = [k0 (+ 1 if u0 is inside
// tile k0), kb), k0 = the tile of u0 (0 when u0 <= t_grid).
__host__ __device__ inline void ss_window_tiles(long long t_grid, long long kb, long long L, bool horner,
                                                long long tile, long long* a, long long* b) {
  const long long u0 = t_grid + tile * kb - 2 * L - (horner ? 1 : 0);
  long long k0 = 0;
  bool partial = false;
  if (u0 > t_grid) {
    k0 = (u0 - t_grid) / tile;
    partial = u0 > t_grid + tile * k0;
  }
  *a = k0 + (partial ? 1 : 0);
  *b = kb;
}

// Appends the row's work items to out (if not null) and returns their number; *slots is advanced by
// the number of look-back slots the row uses, *subtiles by the sub-tiles it processes.
__host__ __device__ inline long long row_work(const RowSpec& r, long long T, WorkItem* out, long long* slots,
                                              long long* subtiles, bool* chained) {
  // stored output positions: [D, D + N), or the row's window (a padded row stores its centre only)
  const long long t_first_out = r.o_hi > 0 ? r.o_lo : r.D, t_last_out = r.o_hi > 0 ? r.o_hi : r.D + r.N;
  const bool short_window = 2 * r.L <= 2 * T;
  long long n = 0;
  *chained = !(short_window && r.policy != SEG_PLAIN);
  long long R;  // outputs per segment
  if (!*chained) {
    // CTA windows: ceil(10 L / T) sub-tiles; warp windows: max(2, ceil(seg_mult L / WT)) warp-tiles,
    // i.e. a prologue of at most about 2 / seg_mult of the segment
    long long sub = r.warp_window ? (r.seg_mult * r.L + r.wt - 1) / r.wt : (10 * r.L + r.wt - 1) / r.wt;
    if (sub < (r.warp_window ? 2 : 1)) sub = r.warp_window ? 2 : 1;
    R = sub * r.wt - 2 * r.L - (r.align - 1);  // room for rounding the segment start down to 32 bytes
  } else if (r.policy == SEG_RESTART) {
    R = 4 * T > 4 * r.L ? 4 * T : 4 * r.L;
  } else {
    R = r.N;
  }
  if (R < 1) R = 1;
  for (long long ts = t_first_out; ts < t_last_out; ts += R) {
    const long long te = (ts + R < t_last_out) ? ts + R : t_last_out;
    const long long t_dom = (ts - 2 * r.L > 0) ? ts - 2 * r.L : 0;
    // first processed position: t_dom rounded down so that the lead loads start 32-byte aligned
    long long t_a = t_dom - ((((r.x_off + t_dom) % r.align) + r.align) % r.align);
    const long long step = *chained ? T : r.wt;
    const long long n_tiles = (te - t_a + step - 1) / step;
    if (!*chained) {
      if (out) {
        WorkItem w{};
        w.x_off = r.x_off;
        w.n = r.N;
        w.out_off = r.out_off;
        w.scale = r.scale;
        w.chain = r.chain;
        w.n_sub = (int)n_tiles;
        w.t_a = t_a;
        w.t_dom = t_dom;
        w.t_out = ts;
        w.t_end = te;
        w.slot = -1;
        w.slot_first = -1;
        w.p_row = -1;
        out[n] = w;
      }
      ++n;
      *subtiles += n_tiles;
    } else {
      const long long first = *slots;
      for (long long k = 0; k < n_tiles; ++k) {
        if (out) {
          WorkItem w{};
          w.x_off = r.x_off;
          w.n = r.N;
          w.out_off = r.out_off;
          w.scale = r.scale;
          w.chain = r.chain;
          w.n_sub = 1;
          w.t_a = t_a + k * T;
          w.t_dom = t_dom;
          w.t_out = ts;
          w.t_end = te;
          w.slot = *slots;
          w.slot_first = first;
          w.p_row = -1;
          out[n] = w;
        }
        ++n;
        ++*slots;
      }
      *subtiles += n_tiles;
    }
  }
  return n;
}

}  // namespace msft
