// Host side of the C ABI (include/morlet_sft.h): plan construction, tile tables, launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/morlet_sft.h"
#include "plan_internal.h"
#include "work_plan.h"

namespace msft {
#define MSFT_DECL(n) const void* n(int); const void* n##_w(int);
MSFT_DECL(kernel_rf_f32c_morlet)
MSFT_DECL(kernel_rf_f32p_morlet)
MSFT_DECL(kernel_rf_f32p_asft)
MSFT_DECL(kernel_rf_f32p_asft_real)
MSFT_DECL(kernel_rf_f32p_mult)
MSFT_DECL(kernel_rf_f64_morlet)
MSFT_DECL(kernel_rf_f32c_real)
MSFT_DECL(kernel_rf_f32p_real)
MSFT_DECL(kernel_rf_f64_real)
#undef MSFT_DECL
const void* kernel_ki_f32c_morlet(int);
const void* kernel_ki_f32p_morlet(int);
const void* kernel_ki_f64_morlet(int);

// The look-back (CTA) kernel of a variant, or with warp = true its warp-independent kernel
// (rotating-form variants only).
const void* kernel_for(int variant, int K, bool warp) {
  switch (variant) {
    case V_RF_F32C_MORLET: return warp ? kernel_rf_f32c_morlet_w(K) : kernel_rf_f32c_morlet(K);
    case V_RF_F32P_MORLET: return warp ? kernel_rf_f32p_morlet_w(K) : kernel_rf_f32p_morlet(K);
    case V_RF_F32P_ASFT: return warp ? kernel_rf_f32p_asft_w(K) : kernel_rf_f32p_asft(K);
    case V_RF_F32P_ASFT_REAL: return warp ? kernel_rf_f32p_asft_real_w(K) : kernel_rf_f32p_asft_real(K);
    case V_RF_F32P_MULT: return warp ? kernel_rf_f32p_mult_w(K) : kernel_rf_f32p_mult(K);
    case V_RF_F64_MORLET: return warp ? kernel_rf_f64_morlet_w(K) : kernel_rf_f64_morlet(K);
    case V_KI_F32C_MORLET: return warp ? nullptr : kernel_ki_f32c_morlet(K);
    case V_KI_F32P_MORLET: return warp ? nullptr : kernel_ki_f32p_morlet(K);
    case V_KI_F64_MORLET: return warp ? nullptr : kernel_ki_f64_morlet(K);
    case V_RF_F32C_REAL: return warp ? kernel_rf_f32c_real_w(K) : kernel_rf_f32c_real(K);
    case V_RF_F32P_REAL: return warp ? kernel_rf_f32p_real_w(K) : kernel_rf_f32p_real(K);
    case V_RF_F64_REAL: return warp ? kernel_rf_f64_real_w(K) : kernel_rf_f64_real(K);
    default: return nullptr;
  }
}
}  // namespace msft

using namespace msft;

namespace {

constexpr int ITEMS = 16;
constexpr long long TILE = (long long)THREADS * ITEMS;
constexpr long long DEFAULT_SPIN = 1LL << 20;  // polls of ~64 ns sleep + an L2 round trip: about 1 s
// work counters per launch: look-back kernel, warp kernel (window items), warp kernel (start-state
// items), prefix-sum kernel, lane-chunk kernel
constexpr int TICKETS = 5;
constexpr long long PS_TILE_H = 512, PS_CHUNK_H = 8;  // prefix-sum tile and chunk (psum_kernel.cuh)
constexpr long long TS_CHUNK_H = 8;                    // tiles per tile-sum work item
// Rows whose half window exceeds this start their work items from exact states (window sums of
// tile sums, or prefix sums); the default, without autotuning. A window segment restarts 2L
// positions before its first output and runs about 16 L positions, so its FP32 residue history
// grows with L; for L > 2048 a resonant input (a chirp through the kernel's band) takes it past
// 1e-5 of max|W| (1.4e-5 measured at L = 4096), while start-state items (up to 64 warp-tiles from
// an exact state, two-float carries between warp-tiles) stay within the gate at any L. Lower
// thresholds, down to 1 (start-state items for every row), are the autotuner's to choose.
constexpr long long SS_MIN_L = 2048;
// Largest start-state threshold and lane-chunk threshold that keep every row within the
// compensated-FP32 gate (measured on chirps and white noise, K = 3..6).
constexpr long long SS_MIN_L_MAX = 2048;
constexpr long long LS_MAX_L_MAX = 256;
// Rows whose half window is at most this go to the lane-chunk scan (one pass per sample, a
// prologue of 2L per lane chunk of max(1024, 8 L) positions).
constexpr long long LS_MAX_L = 128;
constexpr int LS_STEP_H = 16;     // positions per lane step of the lane-chunk scan (lscan_kernel.cuh)
constexpr int LS_THREADS_H = 128;  // threads per CTA of the lane-chunk scan (4 warps, lscan_kernel.cuh)

// A launchable transform: kernel, work table, chains and status arrays.
struct Launch {
  const void* func = nullptr;    // look-back (CTA) kernel: chain items, or every item of a KI plan
  const void* func_w = nullptr;  // warp-independent kernel for window items (rotating form)
  WorkItem* d_work = nullptr;
  long long n_work = 0;
  ChainDesc* d_chains = nullptr;
  int grid = 0;
  int grid_w = 0;
  long long sub_tiles = 0;
  long long rows_chain = 0, rows_halo = 0;
  long long chain_end = 0;             // look-back items come first, [0, chain_end)
  const ScaleTab* tabs = nullptr;      // the scales the rows refer to (the adjoint's 2S virtual scales)
  long long n_x = 0;                   // elements of the input buffer the rows read
  // start-state rows (forward, compensated FP32, long windows): warp-kernel items [ss_begin, n_work)
  // start from the prefix sums that the psum kernel computes over the work items d_pwork
  long long ss_begin = 0;
  const void* func_p = nullptr;
  WorkItem* d_pwork = nullptr;
  long long n_pwork = 0;
  int grid_p = 0;
  long long n_pslots = 0, n_ptiles = 0, rows_ss = 0;
  int ss_window = 0;  // start states from window sums of tile sums (tsum kernel) instead of prefix sums
  // start-state workspace: prefix-sum status flags, aggregates and inclusive values, and the prefix
  // sums (or tile sums) at tile ends
  uint32_t* d_pflags = nullptr;
  void* d_pagg = nullptr;
  void* d_pincl = nullptr;
  void* d_pbuf = nullptr;
  // lane-chunk rows (forward, compensated FP32 Morlet, short windows): items d_lwork
  const void* func_l = nullptr;
  WorkItem* d_lwork = nullptr;
  long long n_lwork = 0;
  int grid_l = 0;
  long long rows_lane = 0;
  int32_t l_chunks[4] = {0, 0, 0, 0};  // the most frequent chunk lengths of the items (TMA maps)
};

}  // namespace

struct morlet_plan_s {
  int device = 0;
  int sms = 0;
  morlet_plan_desc desc{};
  std::vector<int64_t> lengths;
  std::vector<double> sigmas;
  std::vector<int64_t> x_off;
  long long n_in = 0;  // input samples of the batch (sum of lengths)
  long long n_pl = 0;  // adjoint: elements per plane (n_in rounded up to a multiple of 4: 16-byte plane starts)
  // MORLET_FLAG_EDGE: every signal copied into a buffer with `pad` replicated edge samples on each
  // side; the rows run on that buffer and store only their centre
  long long pad = 0;
  std::vector<int64_t> xp_off;
  long long n_xpad = 0;
  void* d_xpad = nullptr;
  int64_t* d_pad_desc = nullptr;  // per signal: x_off, xp_off, N
  int K_fit = 0;     // terms per scale after the fit (max over scales)
  int K_kernel = 0;  // compiled term count used
  int form = 2;
  size_t elem = 4;   // bytes per real sample
  ScaleTab* d_tabs = nullptr;
  FitJob* d_jobs = nullptr;
  float2* d_phase = nullptr;  // kernel-integral form: per-scale phase tables
  std::vector<ScaleTab> h_tabs;
  Launch fwd, adj;
  uint32_t* d_flags = nullptr;
  void* d_agg = nullptr;
  void* d_incl = nullptr;
  long long n_slots = 0;
  int nt_slot = 0;               // complex carry values per look-back slot
  // adjoint (morlet_backward): the real and imaginary planes of gW as real signals at 2S virtual
  // scales (q = 2s: weights (cM, 0); q = 2s + 1: (0, -cL), rotating-form tables), their real
  // transforms, one plane per virtual scale, and the descriptors the split kernel reads
  std::vector<ScaleTab> h_tabs_adj;
  ScaleTab* d_tabs_adj = nullptr;
  void* d_gplanes = nullptr;
  void* d_wplanes = nullptr;
  int64_t* d_sig_desc = nullptr;  // per signal: x_off, N
  cudaGraphExec_t gexec_b = nullptr;
  const void* gb_in = nullptr;
  void* gb_out = nullptr;
  long long ss_min_L = 0;        // rows with L above this use start states (0: none)
  long long ls_max_L = 0;        // rows with L up to this use the lane-chunk scan (0: none)
  long long h_ss_min_L = 4096;   // Horner plans (ASFT, multiplication method): rows with L above this
                                 // start from Horner tile-sum states (the rest: window segments)
  // schedule knobs (MORLET_FLAG_AUTOTUNE or morlet_plan_set_schedule); none changes the transform
  int seg_mult = 16;             // window segments of about seg_mult * L positions
  long long ss_tiles_max = 32;   // start-state items of at most this many 512-position tiles
  int order = 0;                 // 0: scales in index order inside a signal block; 1: decreasing L;
                                 // 2: order 0, then the items of each launch longest first
  int asft_chains = 0;           // ASFT: 1 = one look-back chain per row, 0 = window segments (L <= 4096)
  int tuned = 0;                 // 1: the autotuner ran; -1: it was skipped (no scratch memory)
  long long tune_outputs = 0;    // outputs of the rows the autotuner timed
  unsigned long long* d_ticket = nullptr;  // TICKETS counters per launch (adjoint: per scale)
  int* h_err = nullptr;                    // host-mapped error word
  int* d_err = nullptr;
  long long spin = DEFAULT_SPIN;
  long long skip_tickets = 0;
  int latched = 0;
  cudaStream_t aux = nullptr;  // second stream: the warp-independent kernel runs beside the look-back one
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // graph of the forward (memsets + kernels) for a given (x, W)
  cudaGraphExec_t gexec = nullptr;
  const void* g_x = nullptr;
  void* g_out = nullptr;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MORLET_OK;
  if (e == cudaErrorMemoryAllocation) return MORLET_ERR_NOMEM;
  return MORLET_ERR_CUDA;
}

#define CK(call)                         \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) {             \
      rc = cuda_status(e_);              \
      goto fail;                         \
    }                                    \
  } while (0)

int round_k(int K) {
  for (int i = 0; i < N_KBUILT; ++i)
    if (kbuilt(i) >= K) return kbuilt(i);
  return -1;
}

int variant_of(const morlet_plan_s* p, bool adjoint) {
  const int prec = p->desc.precision;
  // the adjoint runs real-output rotating-form rows on the planes of gW
  if (adjoint) return prec == MORLET_FP64 ? V_RF_F64_REAL : prec == MORLET_FP32_COMP ? V_RF_F32C_REAL : V_RF_F32P_REAL;
  if (p->desc.method == MORLET_MULTIPLY) return V_RF_F32P_MULT;
  if (p->desc.method == MORLET_GAUSS) {
    if (p->desc.transform == MORLET_ASFT) return V_RF_F32P_ASFT_REAL;
    return prec == MORLET_FP64 ? V_RF_F64_REAL : prec == MORLET_FP32_COMP ? V_RF_F32C_REAL : V_RF_F32P_REAL;
  }
  if (p->desc.transform == MORLET_ASFT) return V_RF_F32P_ASFT;
  if (p->form == 1)
    return prec == MORLET_FP64 ? V_KI_F64_MORLET : prec == MORLET_FP32_COMP ? V_KI_F32C_MORLET : V_KI_F32P_MORLET;
  return prec == MORLET_FP64 ? V_RF_F64_MORLET : prec == MORLET_FP32_COMP ? V_RF_F32C_MORLET : V_RF_F32P_MORLET;
}

long long floordiv(long long a, long long b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

// Work table of one transform. Rows are (signal, scale) pairs taken in `order`; each row is cut
// into segments by row_work (work_plan.h), which explains the precision policies.
int seg_policy(const morlet_plan_s* p) {
  if (p->desc.method == MORLET_MULTIPLY) return SEG_RESTART;  // window segments (L <= 4096), start states beyond
  if (p->desc.flags & MORLET_FLAG_NO_HALO) return SEG_PLAIN;
  // The damped ASFT forgets its rounding history, so it needs no restarts: short windows go to window
  // segments like every other row, long windows keep one look-back chain per row (a restart would
  // recompute a 2L prologue per segment for nothing). The schedule may instead put every ASFT row on
  // one chain (fewer, longer work units: better for small batches of long windows).
  if (p->desc.transform == MORLET_ASFT) return p->asft_chains ? SEG_PLAIN : SEG_ROW;
  if (p->desc.precision == MORLET_FP32_PLAIN) return SEG_PLAIN;
  if (p->desc.precision == MORLET_FP32_COMP && p->desc.transform == MORLET_SFT) return SEG_RESTART;
  return SEG_ROW;
}

// Plans whose long-window rows start from window sums of Horner tile sums: the ASFT (damped rho)
// unless the schedule puts its rows on chains, and the multiplication method (non-harmonic rho).
// Plans whose long rows can start from Horner tile-sum states (ASFT, multiplication method; FP32,
// rotating form, no forced chains), whatever the ASFT's chain policy.
bool horner_capable(const morlet_plan_s* p) {
  if (p->form != 2 || p->desc.precision == MORLET_FP64 || (p->desc.flags & MORLET_FLAG_NO_HALO)) return false;
  return p->desc.method == MORLET_MULTIPLY || p->desc.transform == MORLET_ASFT;
}

bool horner_plan(const morlet_plan_s* p) {
  if (p->form != 2 || p->desc.precision == MORLET_FP64 || (p->desc.flags & MORLET_FLAG_NO_HALO)) return false;
  return p->desc.method == MORLET_MULTIPLY || (p->desc.transform == MORLET_ASFT && !p->asft_chains);
}

// Start-state rows (forward, real input, rotating form, long window):
//  - the compensated FP32 SFT with L > ss_min_L (window sums of Reinsch tile sums, or prefix sums);
//  - Horner plans with 2L > 2T, the rows that would otherwise need a look-back chain (their window
//    of 2L + 1 samples summed from FP32 tile sums; the damped sum of the ASFT forgets the tile sums'
//    rounding, the multiplication method's sums carry it like the SFT's window sums do).
bool ss_row(const morlet_plan_s* p, bool adjoint, const ScaleTab& tb) {
  // the adjoint's rows are compensated (or plain, or FP64) real-output SFT rows in the rotating form
  if (adjoint)
    return p->ss_min_L > 0 && p->desc.precision == MORLET_FP32_COMP && !(p->desc.flags & MORLET_FLAG_NO_HALO) &&
           tb.L > p->ss_min_L;
  if (horner_plan(p)) return tb.L > p->h_ss_min_L;
  return p->ss_min_L > 0 && p->form == 2 && p->desc.precision == MORLET_FP32_COMP &&
         p->desc.transform == MORLET_SFT && p->desc.method != MORLET_MULTIPLY &&
         !(p->desc.flags & MORLET_FLAG_NO_HALO) && tb.L > p->ss_min_L;
}

// Lane-chunk rows: forward, compensated FP32 SFT Morlet in the rotating form, short window.
// (Positions inside such a row are 32-bit in the kernel: rows stay below 2^30 positions.)
bool ls_row(const morlet_plan_s* p, bool adjoint, const ScaleTab& tb, long long N) {
  return !adjoint && p->ls_max_L > 0 && p->form == 2 && p->desc.precision == MORLET_FP32_COMP &&
         p->desc.transform == MORLET_SFT && p->desc.method == MORLET_DIRECT &&
         !(p->desc.flags & MORLET_FLAG_NO_HALO) && tb.L <= p->ls_max_L && N + 2 * tb.L + (1LL << 20) < (1LL << 30);
}

// Tiles of a start-state row: tile 0 starts at t_grid (the input element of every tile start is
// 32-byte aligned); the stored outputs (positions [o_lo, o_hi)) lie in tiles [kD, kE].
void ss_tiles(long long x_off, long long o_lo, long long o_hi, long long& t_grid, long long& kD, long long& kE) {
  const long long g = (8 - (x_off % 8)) % 8;
  t_grid = g - PS_TILE_H;
  kD = (o_lo - t_grid) / PS_TILE_H;
  kE = (o_hi - 1 - t_grid) / PS_TILE_H;
}

void build_work(const morlet_plan_s* p, bool adjoint, std::vector<WorkItem>& work, std::vector<ChainDesc>& chains,
                long long& slots, Launch& ln, std::vector<WorkItem>& pwork, std::vector<WorkItem>& lwork,
                long long warp_slots) {
  // Forward: the S scales. Adjoint: 2S virtual scales q, the real (q = 2s) and imaginary (q = 2s + 1)
  // plane of gW at scale s, each row reading and writing plane q (planes of n_pl elements).
  const int S = adjoint ? 2 * (int)p->sigmas.size() : (int)p->sigmas.size();
  const std::vector<ScaleTab>& tabs = adjoint ? p->h_tabs_adj : p->h_tabs;
  const long long nsig = (long long)p->lengths.size();
  // Row order: blocks of signals holding about 16 M input samples, scale by scale inside a block, so
  // that a block's samples are mostly served from L2 to its later scales. With p->order = 1 the scales
  // of a block go in decreasing L, so that the last items claimed are the short ones.
  std::vector<int> sorder(S);
  for (int s = 0; s < S; ++s) sorder[s] = s;
  if (p->order == 1)
    std::stable_sort(sorder.begin(), sorder.end(), [&tabs](int a, int b) { return tabs[a].L > tabs[b].L; });
  std::vector<std::pair<long long, int>> order;  // (signal, scale)
  {
    long long b0 = 0;
    while (b0 < nsig) {
      long long b1 = b0, acc = 0;
      while (b1 < nsig && (b1 == b0 || acc + p->lengths[b1] <= (16LL << 20))) acc += p->lengths[b1++];
      for (int q = 0; q < S; ++q)
        for (long long i = b0; i < b1; ++i) order.push_back({i, sorder[q]});
      b0 = b1;
    }
  }
  const int esz = (int)p->elem;  // bytes per input element
  const long long E = adjoint ? 0 : p->pad;
  // the row (signal i, scale s): first input element, first output element
  auto row_in = [&](long long i, int s) -> long long {
    if (adjoint) return (long long)s * p->n_pl + p->x_off[i];
    return E ? p->xp_off[i] : p->x_off[i];
  };
  auto row_out = [&](long long i, int s) -> long long {
    if (adjoint) return (long long)s * p->n_pl + p->x_off[i];
    return (long long)S * p->x_off[i] + (long long)s * p->lengths[i] - E;  // scalogram row (minus the pad)
  };
  // start-state items: n_ss tiles each, as many tiles as leaves about four items per warp slot
  long long ss_total = 0;
  for (auto& rs : order) {
    const ScaleTab& tb = tabs[rs.second];
    if (!ss_row(p, adjoint, tb)) continue;
    long long tg, kD, kE;
    ss_tiles(row_in(rs.first, rs.second), tb.D + E, tb.D + E + p->lengths[rs.first], tg, kD, kE);
    ss_total += kE - kD + 1;
  }
  const long long n_ss = std::max(4LL, std::min(p->ss_tiles_max, ss_total / std::max(1LL, 4 * warp_slots)));
  // A start state costs a window sum over its 2L / 512 tiles: cheap next to an item of n_ss tiles
  // unless the window is much longer; then the prefix sums (one chained pass) are used instead.
  long long max_win = 0;
  for (auto& rs : order)
    if (ss_row(p, adjoint, tabs[rs.second])) max_win = std::max<long long>(max_win, 2 * tabs[rs.second].L / PS_TILE_H + 2);
  ln.ss_window = ((!adjoint && horner_plan(p)) || max_win <= 16 * n_ss) ? 1 : 0;  // Horner rows: window sums only
  const bool horner_rows = !adjoint && horner_plan(p);
  for (auto& rs : order) {
    const long long i = rs.first;
    const int s = rs.second;
    const ScaleTab& tb = tabs[s];
    const long long N0 = p->lengths[i];
    // edge mode: the row is the padded signal (N0 + 2E samples) and stores positions
    // [D + E, D + E + N0), i.e. the outputs of the original samples
    const long long N = N0 + 2 * E;
    const long long o_lo = tb.D + E, o_hi = tb.D + E + N0;
    ChainDesc c{};
    c.n = N;
    c.x_off = row_in(i, s);
    c.out_off = row_out(i, s);
    c.scale = s;
    const int ci = (int)chains.size();
    chains.push_back(c);
    if (ls_row(p, adjoint, tb, N)) {
      // 32 lane chunks of C positions per item, each after a prologue of >= 2L positions; chunks
      // start where the output element is a multiple of 4 (32-byte stores), the first one possibly
      // up to three positions before D (its outputs there are masked)
      const long long Cfull = std::min<long long>(4096, std::max<long long>(1024, (8 * tb.L + LS_STEP_H - 1) / LS_STEP_H * LS_STEP_H));
      const long long pro = (2 * tb.L + LS_STEP_H - 1) / LS_STEP_H * LS_STEP_H;
      const long long t_first = o_lo, t_last = o_hi;
      const long long e0 = c.out_off + (t_first - tb.D);  // output element of t_first
      long long s0 = t_first - (((e0 % 4) + 4) % 4);
      while (s0 < t_last) {
        const long long rem = t_last - s0;
        long long Ci = Cfull;
        if (rem < 32 * Cfull) Ci = std::max<long long>(LS_STEP_H, ((rem + 31) / 32 + LS_STEP_H - 1) / LS_STEP_H * LS_STEP_H);
        WorkItem w{};
        w.x_off = c.x_off;
        w.n = N;
        w.out_off = c.out_off;
        w.scale = s;
        w.chain = ci;
        w.n_sub = (int)Ci;
        w.t_a = s0;
        w.t_dom = pro;
        w.t_out = t_first;
        w.t_end = t_last;
        w.slot = -1;
        w.slot_first = -1;
        w.p_row = -1;
        lwork.push_back(w);
        ln.sub_tiles += (32 * (Ci + pro) + 511) / 512;
        s0 += 32 * Ci;
      }
      ln.rows_lane++;
      continue;
    }
    if (ss_row(p, adjoint, tb)) {
      long long tg, kD, kE;
      ss_tiles(c.x_off, o_lo, o_hi, tg, kD, kE);
      const long long pbase = ln.n_ptiles;
      long long k_last = kD;  // tile of the last item start
      for (long long k = kD; k <= kE; k += n_ss) {
        const long long nsub = std::min(n_ss, kE - k + 1);
        WorkItem w{};
        w.x_off = c.x_off;
        w.n = N;
        w.out_off = c.out_off;
        w.scale = s;
        w.chain = ci;
        w.n_sub = (int)nsub;
        w.t_a = tg + PS_TILE_H * k;
        w.t_dom = 0;
        w.t_out = std::max<int64_t>(w.t_a, o_lo);
        w.t_end = std::min<int64_t>(w.t_a + PS_TILE_H * nsub, o_hi);
        w.slot = -1;
        w.slot_first = -1;
        w.p_row = pbase;
        w.t_grid = tg;
        work.push_back(w);
        ln.sub_tiles += nsub;
        k_last = k;
      }
      // Prefix sums at the ends of tiles 0 .. k_last - 1 (prefix mode: every tile); or tile sums
      // (window mode) of the tiles the item starts kb read (ss_window_tiles), in chunks.
      const long long n_t = k_last;
      const long long first = ln.n_pslots;
      const long long chunk = ln.ss_window ? TS_CHUNK_H : PS_CHUNK_H;
      std::vector<std::pair<long long, long long>> need;  // tile ranges [a, b)
      if (ln.ss_window) {
        for (long long kb = kD; kb <= k_last; kb += n_ss) {
          long long a, b;
          ss_window_tiles(tg, kb, tb.L, horner_rows, PS_TILE_H, &a, &b);
          if (a >= b) continue;
          if (!need.empty() && a <= need.back().second) need.back().second = std::max(need.back().second, b);
          else need.push_back({a, b});
        }
      } else {
        need.push_back({0, n_t});
      }
      for (auto& rg : need) {
        for (long long k = rg.first; k < rg.second; k += chunk) {
          WorkItem w{};
          w.x_off = c.x_off;
          w.n = N;
          w.out_off = c.out_off;
          w.scale = s;
          w.chain = ci;
          w.n_sub = (int)std::min(chunk, rg.second - k);
          w.t_a = tg + PS_TILE_H * k;
          w.slot = ln.n_pslots++;
          w.slot_first = first;
          w.p_row = pbase + k;
          w.t_grid = tg;
          pwork.push_back(w);
        }
      }
      ln.n_ptiles += n_t;
      ln.rows_ss++;
      continue;
    }
    const bool warp_window = adjoint || p->form != 1;  // the adjoint's rows are rotating-form rows
    const RowSpec r = make_row_spec(N, tb.L, tb.D, c.x_off, c.out_off, s, esz, seg_policy(p), ci, warp_window,
                                    TILE, o_lo, o_hi, p->seg_mult);
    long long sl = slots, st = 0;
    bool chained = false;
    const long long n = row_work(r, TILE, nullptr, &sl, &st, &chained);
    const size_t at = work.size();
    work.resize(at + n);
    ln.sub_tiles += st;
    st = 0;
    row_work(r, TILE, work.data() + at, &slots, &st, &chained);
    if (chained) ln.rows_chain++;
    else ln.rows_halo++;
  }
  // Put the look-back items first (stable), so that independent items may claim their successor ticket
  // early without ever holding an item that others wait on; then the window items, then the
  // start-state items (which wait for the prefix or tile sums).
  auto mid = std::stable_partition(work.begin(), work.end(), [](const WorkItem& w) { return w.slot >= 0; });
  ln.chain_end = (long long)(mid - work.begin());
  auto ss = std::stable_partition(mid, work.end(), [](const WorkItem& w) { return w.p_row < 0; });
  ln.ss_begin = (long long)(ss - work.begin());
  if (p->order == 2) {
    // longest items first inside each launch, so that the last items claimed are short ones and the
    // launch ends with few warps idle (independent items only; look-back items keep their order)
    auto longer = [](const WorkItem& a, const WorkItem& b) { return a.n_sub > b.n_sub; };
    std::stable_sort(mid, ss, longer);
    std::stable_sort(ss, work.end(), longer);
    std::stable_sort(lwork.begin(), lwork.end(),
                     [](const WorkItem& a, const WorkItem& b) { return a.n_sub + a.t_dom > b.n_sub + b.t_dom; });
  }
}

int setup_launch(morlet_plan_s* p, bool adjoint, Launch& ln, long long& slots) {
  int rc = MORLET_OK;
  std::vector<WorkItem> work, pwork, lwork;
  std::vector<ChainDesc> chains;
  ln.func = kernel_for(variant_of(p, adjoint), p->K_kernel, false);
  if (!ln.func) return MORLET_ERR_UNSUPPORTED;
  ln.tabs = adjoint ? p->d_tabs_adj : p->d_tabs;
  ln.n_x = adjoint ? 2 * (long long)p->sigmas.size() * p->n_pl : (p->pad > 0 ? p->n_xpad : p->n_in);
  if (adjoint || p->form != 1) {
    ln.func_w = kernel_for(variant_of(p, adjoint), p->K_kernel, true);
    if (!ln.func_w) return MORLET_ERR_UNSUPPORTED;
    int occw = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occw, ln.func_w, THREADS, 0));
    if (occw < 1) occw = 1;
    ln.grid_w = occw * p->sms;
  }
  build_work(p, adjoint, work, chains, slots, ln, pwork, lwork, (long long)ln.grid_w * WARPS);
  ln.n_work = (long long)work.size();
  // the multiplication method's combine (separate weights for the imaginary part) is built into the
  // warp kernel only: its rows are window segments or start-state items, never look-back chains
  if (p->desc.method == MORLET_MULTIPLY && ln.rows_chain > 0) return MORLET_ERR_UNSUPPORTED;
  {
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ln.func, THREADS, 0));
    if (occ < 1) occ = 1;
    ln.grid = (int)std::min<long long>((long long)occ * p->sms, std::max<long long>(1, ln.n_work));
  }
  if (!pwork.empty()) {
    ln.func_p = (!adjoint && horner_plan(p)) ? kernel_tsum_h(p->K_kernel)
                : ln.ss_window ? kernel_tsum(p->K_kernel) : kernel_psum(p->K_kernel);
    if (!ln.func_p) return MORLET_ERR_UNSUPPORTED;
    int occp = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occp, ln.func_p, THREADS, 0));
    if (occp < 1) occp = 1;
    ln.grid_p = occp * p->sms;
    ln.n_pwork = (long long)pwork.size();
    CK(cudaMalloc(&ln.d_pwork, sizeof(WorkItem) * pwork.size()));
    CK(cudaMemcpy(ln.d_pwork, pwork.data(), sizeof(WorkItem) * pwork.size(), cudaMemcpyHostToDevice));
  }
  if (!lwork.empty()) {
    ln.func_l = kernel_lscan(p->K_kernel);
    if (!ln.func_l) return MORLET_ERR_UNSUPPORTED;
    int occl = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occl, ln.func_l, LS_THREADS_H, 0));
    if (occl < 1) occl = 1;
    ln.grid_l = occl * p->sms;
    ln.n_lwork = (long long)lwork.size();
    {
      std::map<int32_t, long long> cnt;
      for (const auto& it : lwork) cnt[it.n_sub]++;
      std::vector<std::pair<long long, int32_t>> by(cnt.size());
      size_t u = 0;
      for (const auto& c : cnt) by[u++] = {c.second, c.first};
      std::sort(by.begin(), by.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
      for (size_t q = 0; q < 4 && q < by.size(); ++q) ln.l_chunks[q] = by[q].second;
    }
    CK(cudaMalloc(&ln.d_lwork, sizeof(WorkItem) * lwork.size()));
    CK(cudaMemcpy(ln.d_lwork, lwork.data(), sizeof(WorkItem) * lwork.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMalloc(&ln.d_work, sizeof(WorkItem) * std::max<size_t>(1, work.size())));
  CK(cudaMalloc(&ln.d_chains, sizeof(ChainDesc) * std::max<size_t>(1, chains.size())));
  CK(cudaMemcpy(ln.d_work, work.data(), sizeof(WorkItem) * work.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ln.d_chains, chains.data(), sizeof(ChainDesc) * chains.size(), cudaMemcpyHostToDevice));
  return MORLET_OK;
fail:
  return rc;
}

void free_launch(Launch& ln) {
  cudaFree(ln.d_work);
  cudaFree(ln.d_chains);
  cudaFree(ln.d_pwork);
  cudaFree(ln.d_lwork);
  cudaFree(ln.d_pflags);
  cudaFree(ln.d_pagg);
  cudaFree(ln.d_pincl);
  cudaFree(ln.d_pbuf);
  ln.d_work = nullptr;
  ln.d_chains = nullptr;
  ln.d_pwork = nullptr;
  ln.d_lwork = nullptr;
  ln.d_pflags = nullptr;
  ln.d_pagg = ln.d_pincl = ln.d_pbuf = nullptr;
}

int check_latched(morlet_plan_s* p) {
  if (p->latched) return p->latched;
  if (p->h_err && *(volatile int*)p->h_err) {
    p->latched = MORLET_ERR_TIMEOUT;
    return p->latched;
  }
  return MORLET_OK;
}

size_t carry_bytes(const morlet_plan_s* p) {
  // float2 carries for the plain precision and the ASFT; two-float (DFC) or FP64 complex otherwise
  return (p->desc.precision == MORLET_FP32_PLAIN || p->desc.transform == MORLET_ASFT) ? 8 : 16;
}

// Edge mode: xp[xp_off_i + j] = x[x_off_i + clamp(j - E, 0, N_i - 1)] for j in [0, N_i + 2E) (the
// paper's "values on the edges of the interval" extension, Sec. II).
template <typename T>
__global__ void pad_edges_kernel(const T* __restrict__ x, T* __restrict__ xp, const int64_t* __restrict__ desc,
                                 int64_t nsig, int64_t E) {
  for (int64_t i = blockIdx.y; i < nsig; i += gridDim.y) {
    const int64_t xo = desc[3 * i], po = desc[3 * i + 1], n = desc[3 * i + 2];
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n + 2 * E;
         j += (int64_t)gridDim.x * blockDim.x) {
      int64_t u = j - E;
      u = u < 0 ? 0 : (u >= n ? n - 1 : u);
      xp[po + j] = x[xo + u];
    }
  }
}

cudaError_t pad_edges(const morlet_plan_s* p, const void* x, cudaStream_t st) {
  long long longest = 0;
  for (auto n : p->lengths) longest = std::max<long long>(longest, n + 2 * p->pad);
  const long long nsig = (long long)p->lengths.size();
  const dim3 grid((unsigned)std::min<long long>(1024, (longest + 255) / 256), (unsigned)std::min<long long>(65535, nsig));
  if (p->elem == 8)
    pad_edges_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double*>(x), static_cast<double*>(p->d_xpad),
                                                   p->d_pad_desc, nsig, p->pad);
  else
    pad_edges_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float*>(x), static_cast<float*>(p->d_xpad),
                                                  p->d_pad_desc, nsig, p->pad);
  return cudaGetLastError();
}

// Enqueue one launch: reset its work counters (and the status flags), then
//  - on the plan's second stream, the lane-chunk kernel and the warp kernel over the window items;
//  - on `st`, the prefix-sum (or tile-sum) kernel and after it the warp kernel over the start-state
//    items, then the look-back kernel over the chain items;
// and join the second stream back into `st`. tickets[0..4] count the look-back, window, start-state,
// prefix-sum and lane-chunk kernels. `x` is the buffer the rows read (the forward's input, its padded
// copy in edge mode, or the adjoint's planes), `out` the buffer they write.
// The driver's tensor-map encoder, looked up once (the runtime links no driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    else
      (void)cudaGetLastError();
  });
  return fn;
}

// Tensor maps of an output buffer of `bytes` bytes for the warp scan's TMA stores: map m views the
// buffer from out + 16 m as rows of 32 floats (128 bytes), with boxes of 32 rows and the 128-byte
// swizzle. False (plain stores) when the buffer is not 16-byte aligned, too small to hold a
// warp-tile, too long for 32-bit row coordinates, or the encoder is unavailable.
bool encode_out_maps(KParams& kp, void* out, size_t bytes) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || (reinterpret_cast<uintptr_t>(out) & 15) != 0 || bytes < 4096 + 128) return false;
  for (int m = 0; m < 8; ++m) {
    const cuuint64_t rows = (cuuint64_t)((bytes - 16 * (size_t)m) / 128);
    if (rows >= (1ull << 31)) return false;
    const cuuint64_t dims[2] = {32, rows};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&kp.omap[m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, static_cast<char*>(out) + 16 * m, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

// Tensor maps of the output for the lane-chunk scan's TMA stores: for each chunk length C of
// `chunks` (0: none), the buffer viewed as rows of C complex outputs (8 C bytes), boxes of 32 floats
// (16 outputs) x 32 rows (the 32 lane chunks of an item), 128-byte swizzle. A length whose view has
// fewer than 32 rows, or that fails to encode, gets none (plain stores).
void encode_chunk_maps(KParams& kp, void* out, size_t bytes, const int32_t (&chunks)[4]) {
  const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  for (int q = 0; q < 4; ++q) {
    kp.lmap_c[q] = 0;
    kp.lmap_rows[q] = 0;
    const int32_t c = chunks[q];
    if (!enc || c < 16 || c % 16 != 0 || (reinterpret_cast<uintptr_t>(out) & 15) != 0) continue;
    const cuuint64_t rows = (cuuint64_t)(bytes / (8 * (size_t)c));
    if (rows < 32 || rows >= (1ull << 31)) continue;
    const cuuint64_t dims[2] = {2 * (cuuint64_t)c, rows};
    const cuuint64_t strides[1] = {8 * (cuuint64_t)c};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&kp.lmap[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, out, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      continue;
    kp.lmap_c[q] = c;
    kp.lmap_rows[q] = (int64_t)rows;
  }
}

cudaError_t enqueue(morlet_plan_s* p, const Launch& ln, const void* x, void* out, unsigned long long* tickets,
                    cudaStream_t st) {
  const long long w_end = ln.n_work;
  const bool two = ln.func_w != nullptr;
  const long long c_end = two ? ln.chain_end : w_end;
  const long long s_beg = two ? std::min(std::max(ln.ss_begin, c_end), w_end) : w_end;
  cudaError_t e = cudaMemsetAsync(tickets, 0, TICKETS * sizeof(unsigned long long), st);
  if (e == cudaSuccess && p->skip_tickets > 0) {
    // testing hook: skip the first work items of the first look-back kernel of this launch
    const unsigned long long v = (unsigned long long)p->skip_tickets;
    const int at = (w_end > s_beg && ln.n_pwork > 0 && !ln.ss_window) ? 3 : 0;
    e = cudaMemcpyAsync(tickets + at, &v, sizeof(v), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    p->skip_tickets = 0;
  }
  if (e != cudaSuccess) return e;
  if (c_end > 0 && p->n_slots > 0) {
    e = cudaMemsetAsync(p->d_flags, 0, sizeof(uint32_t) * p->n_slots, st);
    if (e != cudaSuccess) return e;
  }
  KParams kp{};
  kp.x = x;
  kp.out = out;
  kp.chains = ln.d_chains;
  kp.tabs = ln.tabs;
  kp.flags = p->d_flags;
  kp.agg = p->d_agg;
  kp.incl = p->d_incl;
  kp.err = p->d_err;
  kp.spin_limit = p->spin;
  kp.n_x = ln.n_x;
  kp.pbuf = ln.d_pbuf;
  // complex FP32 forward output: whole warp-tiles leave the warp scan, and whole steps the lane-chunk
  // scan, by TMA tensor stores
  if (&ln == &p->fwd && p->elem == 4 && p->desc.method != MORLET_GAUSS) {
    const size_t bytes = sizeof(float2) * p->sigmas.size() * (size_t)p->n_in;
    if (ln.func_w != nullptr) kp.use_tma = encode_out_maps(kp, out, bytes) ? 1 : 0;
    if (ln.n_lwork > 0) encode_chunk_maps(kp, out, bytes, ln.l_chunks);
  }
  bool forked = false;
  const bool lane_items = ln.n_lwork > 0;
  if ((two && s_beg > c_end) || lane_items) {
    e = cudaEventRecord(p->ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->aux, p->ev_fork, 0);
    if (e != cudaSuccess) return e;
    if (lane_items) {
      KParams kl = kp;
      kl.work = ln.d_lwork;
      kl.n_work = ln.n_lwork;
      kl.n_chain = 0;
      kl.ticket = tickets + 4;
      void* args[] = {&kl};
      const int grid = (int)std::min<long long>(ln.grid_l, (kl.n_work + LS_THREADS_H / 32 - 1) / (LS_THREADS_H / 32));
      e = cudaLaunchKernel(ln.func_l, dim3(grid), dim3(LS_THREADS_H), args, 0, p->aux);
      if (e != cudaSuccess) return e;
    }
    if (two && s_beg > c_end) {
      KParams kw = kp;
      kw.work = ln.d_work + c_end;
      kw.n_work = s_beg - c_end;
      kw.n_chain = 0;
      kw.ticket = tickets + 1;
      void* args[] = {&kw};
      const int grid = (int)std::min<long long>(ln.grid_w, (kw.n_work + WARPS - 1) / WARPS);
      e = cudaLaunchKernel(ln.func_w, dim3(grid), dim3(THREADS), args, 0, p->aux);
      if (e != cudaSuccess) return e;
    }
    e = cudaEventRecord(p->ev_join, p->aux);
    if (e != cudaSuccess) return e;
    forked = true;
  }
  if (two && w_end > s_beg) {
    if (ln.n_pwork > 0) {
      if (!ln.ss_window) {
        e = cudaMemsetAsync(ln.d_pflags, 0, sizeof(uint32_t) * ln.n_pslots, st);
        if (e != cudaSuccess) return e;
      }
      KParams kq = kp;
      kq.work = ln.d_pwork;
      kq.n_work = ln.n_pwork;
      kq.n_chain = ln.n_pwork;
      kq.flags = ln.d_pflags;
      kq.agg = ln.d_pagg;
      kq.incl = ln.d_pincl;
      kq.ticket = tickets + 3;
      void* args[] = {&kq};
      const int grid = (int)std::min<long long>(ln.grid_p, (kq.n_work + WARPS - 1) / WARPS);
      e = cudaLaunchKernel(ln.func_p, dim3(grid), dim3(THREADS), args, 0, st);
      if (e != cudaSuccess) return e;
    }
    KParams ks = kp;
    ks.work = ln.d_work + s_beg;
    ks.n_work = w_end - s_beg;
    ks.n_chain = 0;
    ks.ticket = tickets + 2;
    ks.ss_window = ln.ss_window;
    void* args[] = {&ks};
    const int grid = (int)std::min<long long>(ln.grid_w, (ks.n_work + WARPS - 1) / WARPS);
    e = cudaLaunchKernel(ln.func_w, dim3(grid), dim3(THREADS), args, 0, st);
    if (e != cudaSuccess) return e;
  }
  if (c_end > 0) {
    kp.work = ln.d_work;
    kp.n_work = c_end;
    kp.n_chain = std::min(ln.chain_end, c_end);
    kp.ticket = tickets;
    void* args[] = {&kp};
    const int grid = (int)std::min<long long>(ln.grid, kp.n_work);
    e = cudaLaunchKernel(ln.func, dim3(grid), dim3(THREADS), args, 0, st);
    if (e != cudaSuccess) return e;
  }
  if (forked) e = cudaStreamWaitEvent(st, p->ev_join, 0);
  return e;
}

// Workspace of a launch's start-state rows: tile sums (K FP32 complex per tile) in window mode; prefix
// sums (K two-float complex per tile) plus the look-back status, aggregates and inclusive values
// otherwise.
int alloc_prefix(morlet_plan_s* p, Launch& f) {
  int rc = MORLET_OK;
  if (f.ss_window) {
    CK(cudaMalloc(&f.d_pbuf, sizeof(float2) * p->K_kernel * std::max(1LL, f.n_ptiles)));
  } else {
    const size_t kb = sizeof(float4) * p->K_kernel;  // K two-float complex values
    CK(cudaMalloc(&f.d_pflags, sizeof(uint32_t) * f.n_pslots));
    CK(cudaMalloc(&f.d_pagg, kb * f.n_pslots));
    CK(cudaMalloc(&f.d_pincl, kb * f.n_pslots));
    CK(cudaMalloc(&f.d_pbuf, kb * std::max(1LL, f.n_ptiles)));
  }
  return MORLET_OK;
fail:
  return rc;
}

// The adjoint's input: gW [signal][scale][n] (complex) split into its real and imaginary planes,
// plane 2s (real) and 2s + 1 (imaginary) of n_pl elements each, signal i at x_off_i in every plane.
// Each thread moves 4 consecutive samples: 4 independent loads in flight, and for FP32 one 16-byte
// store per plane (samples grouped so that each group starts on a 16-byte plane boundary; the first
// samples of a row, before its first boundary, one by one).
template <typename T>
__global__ void split_planes_kernel(const T* __restrict__ g, T* __restrict__ planes, const int64_t* __restrict__ desc,
                                    int64_t nsig, int32_t S, int64_t n_pl) {
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  for (int64_t r = blockIdx.y; r < nsig * S; r += gridDim.y) {
    const int64_t i = r / S, s = r % S;
    const int64_t xo = desc[2 * i], n = desc[2 * i + 1];
    const T2* gr = reinterpret_cast<const T2*>(g) + (S * xo + s * n);
    T* pa = planes + (2 * s) * n_pl + xo;
    T* pb = pa + n_pl;
    const int64_t h = sizeof(T) == 4 ? (4 - (xo & 3)) & 3 : 0;  // samples before the first boundary
    if (blockIdx.x == 0 && threadIdx.x < h && threadIdx.x < n) {
      const T2 v = __ldcs(gr + threadIdx.x);
      pa[threadIdx.x] = v.x;
      pb[threadIdx.x] = v.y;
    }
    for (int64_t j = h + 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x); j < n;
         j += 4 * (int64_t)gridDim.x * blockDim.x) {
      T2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j + u < n) v[u] = __ldcs(gr + j + u);
      bool done = false;
      if constexpr (sizeof(T) == 4) {
        if (j + 4 <= n) {
          *reinterpret_cast<float4*>(pa + j) = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
          *reinterpret_cast<float4*>(pb + j) = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
          done = true;
        }
      }
      if (!done) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j + u < n) {
            pa[j + u] = v[u].x;
            pb[j + u] = v[u].y;
          }
      }
    }
  }
}

// gx[t] = sum over the nq planes in order (q = 0, 1, ..., nq - 1), so the sum over scales has a fixed
// order (deterministic, no atomics). FP32: 4 consecutive t per thread as 16-byte loads (planes start
// on 16-byte boundaries), 4 planes' loads in flight.
template <typename T>
__global__ void sum_planes_kernel(const T* __restrict__ planes, T* __restrict__ gx, int32_t nq, int64_t n_in,
                                  int64_t n_pl) {
  if constexpr (sizeof(T) == 4) {
    const float4* p4 = reinterpret_cast<const float4*>(planes);
    const int64_t q4 = n_pl / 4;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * g < n_in; g += (int64_t)gridDim.x * blockDim.x) {
      float4 acc = __ldcs(p4 + g);
      int32_t q = 1;
      for (; q + 4 <= nq; q += 4) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcs(p4 + (q + u) * q4 + g);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc.x += v[u].x;
          acc.y += v[u].y;
          acc.z += v[u].z;
          acc.w += v[u].w;
        }
      }
      for (; q < nq; ++q) {
        const float4 v = __ldcs(p4 + q * q4 + g);
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
      }
      const float a[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (4 * g + u < n_in) gx[4 * g + u] = a[u];
    }
  } else {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_in; t += (int64_t)gridDim.x * blockDim.x) {
      T acc = planes[t];
      for (int32_t q = 1; q < nq; ++q) acc += planes[q * n_pl + t];
      gx[t] = acc;
    }
  }
}

// One forward: the edge-padded copy of x first in edge mode, then the launch.
cudaError_t forward_enqueue(morlet_plan_s* p, const void* x, void* W, cudaStream_t st) {
  if (p->pad > 0) {
    const cudaError_t e = pad_edges(p, x, st);
    if (e != cudaSuccess) return e;
    x = p->d_xpad;
  }
  return enqueue(p, p->fwd, x, W, p->d_ticket, st);
}

// One backward: split gW into planes, the real transforms of the 2S planes, the ordered plane sum.
cudaError_t backward_enqueue(morlet_plan_s* p, const void* gW, void* gx, cudaStream_t st) {
  const long long nsig = (long long)p->lengths.size();
  const int S = (int)p->sigmas.size();
  long long longest = 0;
  for (auto n : p->lengths) longest = std::max<long long>(longest, n);
  const dim3 gs((unsigned)std::min<long long>(256, (longest + 1023) / 1024), (unsigned)std::min<long long>(65535, nsig * S));
  const long long groups = p->elem == 4 ? (p->n_in + 3) / 4 : p->n_in;
  const unsigned gr = (unsigned)std::min<long long>(4LL * p->sms * 8, (groups + 255) / 256);
  if (p->elem == 8)
    split_planes_kernel<double><<<gs, 256, 0, st>>>(static_cast<const double*>(gW), static_cast<double*>(p->d_gplanes),
                                                    p->d_sig_desc, nsig, S, p->n_pl);
  else
    split_planes_kernel<float><<<gs, 256, 0, st>>>(static_cast<const float*>(gW), static_cast<float*>(p->d_gplanes),
                                                   p->d_sig_desc, nsig, S, p->n_pl);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = enqueue(p, p->adj, p->d_gplanes, p->d_wplanes, p->d_ticket + TICKETS, st);
  if (e != cudaSuccess) return e;
  if (p->elem == 8)
    sum_planes_kernel<double><<<gr, 256, 0, st>>>(static_cast<const double*>(p->d_wplanes), static_cast<double*>(gx),
                                                  2 * S, p->n_in, p->n_pl);
  else
    sum_planes_kernel<float><<<gr, 256, 0, st>>>(static_cast<const float*>(p->d_wplanes), static_cast<float*>(gx),
                                                 2 * S, p->n_in, p->n_pl);
  return cudaGetLastError();
}

// The forward (or backward) as one CUDA graph (memsets and kernels of both streams), captured once
// per (input, output) pair; replays are a single graph launch.
cudaError_t capture_graph(morlet_plan_s* p, bool backward, const void* in, void* out) {
  cudaGraphExec_t& gx = backward ? p->gexec_b : p->gexec;
  const void*& gin = backward ? p->gb_in : p->g_x;
  void*& gout = backward ? p->gb_out : p->g_out;
  if (gx && gin == in && gout == out) return cudaSuccess;
  if (gx) {
    cudaGraphExecDestroy(gx);
    gx = nullptr;
  }
  cudaStream_t cs;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = backward ? backward_enqueue(p, in, out, cs) : forward_enqueue(p, in, out, cs);
    e = cudaStreamEndCapture(cs, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return e;
  gin = in;
  gout = out;
  return cudaSuccess;
}

cudaError_t forward_graph(morlet_plan_s* p, const void* x, void* W) { return capture_graph(p, false, x, W); }

// Look-back status arrays for n slots (flags, aggregates, inclusive values), replacing the old ones.
int alloc_slots(morlet_plan_s* p, long long n) {
  int rc = MORLET_OK;
  if (p->gexec_b) {  // a captured backward refers to the old arrays
    cudaGraphExecDestroy(p->gexec_b);
    p->gexec_b = nullptr;
  }
  cudaFree(p->d_flags);
  cudaFree(p->d_agg);
  cudaFree(p->d_incl);
  p->d_flags = nullptr;
  p->d_agg = p->d_incl = nullptr;
  p->n_slots = 0;
  if (n > 0) {
    CK(cudaMalloc(&p->d_flags, sizeof(uint32_t) * n));
    CK(cudaMalloc(&p->d_agg, carry_bytes(p) * p->nt_slot * n));
    CK(cudaMalloc(&p->d_incl, carry_bytes(p) * p->nt_slot * n));
    p->n_slots = n;
  }
  return MORLET_OK;
fail:
  return rc;
}

// (Re)build the forward launch and its prefix-sum workspace for the plan's current schedule (row
// thresholds ls_max_L / ss_min_L and the knobs seg_mult, ss_tiles_max, order, asft_chains); grows
// the look-back status arrays if the new schedule needs more slots. Synchronous (frees and
// allocates device memory). `slots` returns the look-back slots the forward needs.
int build_forward(morlet_plan_s* p, long long& slots) {
  int rc = MORLET_OK;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  cudaDeviceSynchronize();
  free_launch(p->fwd);
  p->fwd = Launch{};
  slots = 0;
  rc = setup_launch(p, false, p->fwd, slots);
  if (rc) return rc;
  if (slots > p->n_slots) {
    rc = alloc_slots(p, slots);
    if (rc) return rc;
  }
  if (p->fwd.n_pwork > 0) return alloc_prefix(p, p->fwd);
  return MORLET_OK;
}

// One point of the schedule space.
struct Sched {
  long long ls, ss;   // row thresholds: lane-chunk rows L <= ls, start-state rows L > ss
  int seg_mult;       // window segments of about seg_mult * L positions
  int order;          // scale order inside a signal block
  long long ss_tiles; // start-state item size limit (tiles)
  int asft_chains;    // ASFT rows on one look-back chain each
  long long h_ss;     // Horner plans: start-state rows L > h_ss
};

Sched get_sched(const morlet_plan_s* p) {
  return Sched{p->ls_max_L, p->ss_min_L, p->seg_mult, p->order, p->ss_tiles_max, p->asft_chains, p->h_ss_min_L};
}

void put_sched(morlet_plan_s* p, const Sched& c) {
  p->ls_max_L = c.ls;
  p->ss_min_L = c.ss;
  p->seg_mult = c.seg_mult;
  p->order = c.order;
  p->ss_tiles_max = c.ss_tiles;
  p->asft_chains = c.asft_chains;
  p->h_ss_min_L = c.h_ss;
}

// Compensated FP32 SFT plans in the rotating form (Morlet, Gaussian): the plans with row-kind choices
// (the Gaussian rows have no lane-chunk scan; their limit there has no effect).
bool sft_schedulable(const morlet_plan_s* p) {
  const morlet_plan_desc& d = p->desc;
  return p->form == 2 && d.precision == MORLET_FP32_COMP && d.transform == MORLET_SFT &&
         (d.method == MORLET_DIRECT || d.method == MORLET_GAUSS);
}

constexpr long long TUNE_OUTPUTS = 1LL << 28;  // outputs of the subset the autotuner times when the batch is too big

// MORLET_FLAG_AUTOTUNE: time the forward of this plan's rows under a few schedules and keep the
// fastest. The rows timed are a sub-plan (the same scales and options) with its own scratch input
// and output: the whole batch when that scratch takes at most a quarter of the free device memory
// (the fastest schedule depends on the batch's parallelism: a subset of the signals leaves some
// kernels too few work items), otherwise every k-th signal up to TUNE_OUTPUTS outputs. Each
// candidate is timed as replays of its captured forward graph, the way morlet_forward runs it.
// Knobs are tried set by set, each with the best values of the sets before it:
//  - compensated FP32 SFT Morlet: the row thresholds (13 pairs within the precision limits), the
//    window-segment length (8, 12, 16 L), then the item order (index order, decreasing L, longest
//    items first) together with the start-state item size (16, 32, 64 tiles);
//  - the ASFT: one look-back chain per row against window segments with Horner start states for
//    the rows beyond each window length (4096, 512, 1: every row), then the segment length, that
//    window length again, and the item order together with the start-state item size; the
//    multiplication method the same without the chains.
// Each candidate is timed twice (interleaved passes, the faster kept), and a knob keeps its current
// value unless another is at least 1 % faster. Every schedule computes the same transform. If the
// sub-plan or its scratch buffers cannot be allocated the plan keeps its defaults and reports the
// tuner as skipped (morlet_plan_schedule).
int autotune(morlet_plan_s* p, cudaStream_t st) {
  const morlet_plan_desc& d = p->desc;
  const bool sft = sft_schedulable(p);
  const bool asft = d.transform == MORLET_ASFT && !(d.flags & MORLET_FLAG_NO_HALO);
  const bool mult = d.method == MORLET_MULTIPLY && horner_capable(p);
  if (!sft && !asft && !mult) return MORLET_OK;
  const long long S = (long long)p->sigmas.size();
  const long long nsig = (long long)p->lengths.size();
  const long long total = p->n_in * S;
  const size_t out_elem = (d.method == MORLET_GAUSS ? 1 : 2) * p->elem;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  const bool whole = (double)(out_elem * S + p->elem) * (double)p->n_in <= 0.25 * (double)free_b;
  const long long k = whole ? 1 : std::max(1LL, (total + TUNE_OUTPUTS - 1) / TUNE_OUTPUTS);
  std::vector<int64_t> sub;
  long long acc = 0;
  for (long long i = 0; i < nsig; i += k) {
    if (!whole && !sub.empty() && (acc + p->lengths[i]) * S > TUNE_OUTPUTS) break;
    sub.push_back(p->lengths[i]);
    acc += p->lengths[i];
  }
  morlet_plan_desc sd = d;
  sd.n_signals = (int64_t)sub.size();
  sd.lengths = sub.data();
  sd.sigmas = p->sigmas.data();
  sd.flags = (sd.flags & ~MORLET_FLAG_AUTOTUNE) | MORLET_FLAG_NO_ADJOINT;
  morlet_plan_t q = nullptr;
  int rc = morlet_plan(&q, &sd, st);
  if (rc == MORLET_ERR_NOMEM) {
    cudaGetLastError();
    p->tuned = -1;
    return MORLET_OK;
  }
  if (rc) return rc;
  void* x = nullptr;
  void* W = nullptr;
  if (cudaMalloc(&x, p->elem * std::max(1LL, acc)) != cudaSuccess ||
      cudaMalloc(&W, out_elem * std::max(1LL, acc * S)) != cudaSuccess) {
    cudaFree(x);
    cudaFree(W);
    cudaGetLastError();
    morlet_plan_destroy(q);
    p->tuned = -1;
    return MORLET_OK;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Sched best = get_sched(p);
  float t_best = -1.f;
  // times one schedule on the sub-plan: mean of 3 graph replays after one warm-up; -1 if it cannot run
  auto time_one = [&](const Sched& c, float& ms) -> int {
    ms = -1.f;
    put_sched(q, c);
    long long slots = 0;
    int r = build_forward(q, slots);
    if (r == MORLET_ERR_NOMEM) {
      cudaGetLastError();
      return MORLET_OK;
    }
    if (r) return r;
    cudaError_t e = forward_graph(q, x, W);
    if (e == cudaSuccess) e = cudaGraphLaunch(q->gexec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaGraphLaunch(q->gexec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) return cuda_status(e);
    if (q->h_err && *(volatile int*)q->h_err) {  // a timed-out wait: not a candidate
      *(volatile int*)q->h_err = 0;
      return MORLET_OK;
    }
    ms = t / 3.f;
    return MORLET_OK;
  };
  // tries the candidates (which include the incumbent) in two interleaved passes
  auto try_set = [&](const std::vector<Sched>& cands) -> int {
    std::vector<float> tm(cands.size(), -1.f);
    for (int pass = 0; pass < 2; ++pass)
      for (size_t i = 0; i < cands.size(); ++i) {
        float ms = -1.f;
        const int r = time_one(cands[i], ms);
        if (r) return r;
        if (ms >= 0.f && (tm[i] < 0.f || ms < tm[i])) tm[i] = ms;
      }
    // the incumbent's time in this set, then any candidate at least 1 % faster
    for (size_t i = 0; i < cands.size(); ++i)
      if (memcmp(&cands[i], &best, sizeof(Sched)) == 0 && tm[i] >= 0.f) t_best = tm[i];
    for (size_t i = 0; i < cands.size(); ++i)
      if (tm[i] >= 0.f && (t_best < 0.f || tm[i] < 0.99f * t_best)) {
        best = cands[i];
        t_best = tm[i];
      }
    return MORLET_OK;
  };
  CK(cudaMemsetAsync(x, 0, p->elem * std::max(1LL, acc), st));
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  if (sft) {
    const long long pairs[][2] = {{LS_MAX_L, SS_MIN_L}, {256, SS_MIN_L}, {64, SS_MIN_L}, {0, SS_MIN_L},
                                  {LS_MAX_L, 1024},     {256, 1024},     {64, 1024},       {0, 1024},
                                  {LS_MAX_L, 512},      {256, 512},      {LS_MAX_L, LS_MAX_L}, {64, 64},
                                  {0, 1}};
    std::vector<Sched> c;
    for (auto& pr : pairs) {
      Sched v = best;
      v.ls = pr[0];
      v.ss = pr[1];
      c.push_back(v);
    }
    rc = try_set(c);
    if (rc) goto fail;
    c.clear();
    for (int m : {16, 12, 8}) {
      Sched v = best;
      v.seg_mult = m;
      c.push_back(v);
    }
    rc = try_set(c);
    if (rc) goto fail;
    c.clear();
    // the item order and the start-state item size together: longest-first order pays off with
    // larger items, and neither alone may clear the 1 % margin
    for (int o : {0, 1, 2})
      for (long long t : {32LL, 16LL, 64LL}) {
        Sched v = best;
        v.order = o;
        v.ss_tiles = t;
        c.push_back(v);
      }
    rc = try_set(c);
    if (rc) goto fail;
  } else {
    std::vector<Sched> c;
    if (asft) {  // the multiplication method has no look-back chains
      // one chain per row against window segments with Horner start states from each limit on: the
      // limit decides whether segments win (the c4 Gaussian ASFT batch: chains 79 G outputs/s,
      // segments with the default limit 74, with start states for every row 110)
      for (int a : {0, 1})
        for (long long h : {(long long)TILE, 512LL, 1LL}) {
          if (a == 1 && h != (long long)TILE) continue;
          Sched v = best;
          v.asft_chains = a;
          v.h_ss = a == 1 ? best.h_ss : h;
          c.push_back(v);
        }
      rc = try_set(c);
      if (rc) goto fail;
      c.clear();
    }
    if (!best.asft_chains) {
      for (int m : {16, 12, 8}) {
        Sched v = best;
        v.seg_mult = m;
        c.push_back(v);
      }
      rc = try_set(c);
      if (rc) goto fail;
      c.clear();
      // Horner start states from shorter windows on (1: every row)
      for (long long h : {(long long)TILE, 512LL, 1LL}) {
        Sched v = best;
        v.h_ss = h;
        c.push_back(v);
      }
      rc = try_set(c);
      if (rc) goto fail;
      c.clear();
    }
    for (int o : {0, 1, 2})
      for (long long t : {32LL, 16LL, 64LL}) {
        Sched v = best;
        v.order = o;
        v.ss_tiles = t;
        c.push_back(v);
      }
    rc = try_set(c);
    if (rc) goto fail;
  }
  put_sched(p, best);
  {
    long long slots = 0;
    rc = build_forward(p, slots);
  }
  if (rc == MORLET_OK) {
    p->tuned = 1;
    p->tune_outputs = acc * S;
  }
fail:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(x);
  cudaFree(W);
  morlet_plan_destroy(q);
  return rc;
}

}  // namespace

extern "C" {

const char* morlet_strerror(int status) {
  switch (status) {
    case MORLET_OK: return "ok";
    case MORLET_ERR_ARG: return "invalid argument";
    case MORLET_ERR_UNSUPPORTED: return "unsupported option";
    case MORLET_ERR_CUDA: return "CUDA runtime error";
    case MORLET_ERR_TIMEOUT: return "a kernel timed out waiting for a predecessor tile";
    case MORLET_ERR_NOMEM: return "out of memory";
    default: return "unknown status";
  }
}

void morlet_plan_destroy(morlet_plan_t p) {
  if (!p) return;
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  free_launch(p->fwd);
  free_launch(p->adj);
  cudaFree(p->d_tabs);
  cudaFree(p->d_jobs);
  cudaFree(p->d_xpad);
  cudaFree(p->d_pad_desc);
  cudaFree(p->d_phase);
  cudaFree(p->d_flags);
  cudaFree(p->d_agg);
  cudaFree(p->d_incl);
  cudaFree(p->d_ticket);
  if (p->gexec_b) cudaGraphExecDestroy(p->gexec_b);
  cudaFree(p->d_tabs_adj);
  cudaFree(p->d_gplanes);
  cudaFree(p->d_wplanes);
  cudaFree(p->d_sig_desc);
  if (p->h_err) cudaFreeHost(p->h_err);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->aux) cudaStreamDestroy(p->aux);
  delete p;
}

int morlet_plan(morlet_plan_t* out, const morlet_plan_desc* d, void* stream) {
  if (!out) return MORLET_ERR_ARG;
  *out = nullptr;
  if (!d || d->n_signals < 1 || !d->lengths || d->n_scales < 1 || !d->sigmas) return MORLET_ERR_ARG;
  if (d->K < 0 || d->K > KMAX) return d->K > KMAX ? MORLET_ERR_UNSUPPORTED : MORLET_ERR_ARG;
  if (d->K == 0 && !(d->fit_tol > 0)) return MORLET_ERR_ARG;
  if (d->method != MORLET_DIRECT && d->method != MORLET_GAUSS && d->method != MORLET_MULTIPLY) return MORLET_ERR_ARG;
  // multiplication method: FP32, rotating form, 2K - 1 non-harmonic terms (K Gaussian terms given),
  // plus K harmonic kappa terms for the normalised Morlet (norm = 1); window segments for L <= 4096,
  // start states from window sums of tile sums beyond (no look-back chains)
  if (d->method == MORLET_MULTIPLY &&
      (d->transform != MORLET_SFT || d->precision == MORLET_FP64 || d->form == 1 || d->K < 1 ||
       (d->norm == 1 ? 3 * d->K - 1 : 2 * d->K - 1) > KMAX || (d->flags & MORLET_FLAG_NO_HALO)))
    return MORLET_ERR_UNSUPPORTED;
  if (d->transform != MORLET_SFT && d->transform != MORLET_ASFT) return MORLET_ERR_ARG;
  if (d->precision < MORLET_FP32_PLAIN || d->precision > MORLET_FP64) return MORLET_ERR_ARG;
  if (d->norm != 0 && d->norm != 1) return MORLET_ERR_ARG;
  if (d->form < 0 || d->form > 2) return MORLET_ERR_ARG;
  if (d->method == MORLET_GAUSS && (d->deriv < 0 || d->deriv > 2)) return MORLET_ERR_ARG;
  if (d->transform == MORLET_ASFT && (d->precision == MORLET_FP64 || d->form == 1)) return MORLET_ERR_UNSUPPORTED;
  if (d->n0 < 0 || d->window_mult < 0 || d->spin_limit < 0) return MORLET_ERR_ARG;
  for (int64_t i = 0; i < d->n_signals; ++i)
    if (d->lengths[i] < 1) return MORLET_ERR_ARG;
  for (int32_t s = 0; s < d->n_scales; ++s)
    if (!(d->sigmas[s] >= 0.5) || !(d->sigmas[s] < 1e9)) return MORLET_ERR_ARG;
  if (!(d->xi >= 0.0 && d->xi < 1e6)) return MORLET_ERR_ARG;

  cudaStream_t st = (cudaStream_t)stream;
  morlet_plan_s* p = new (std::nothrow) morlet_plan_s();
  if (!p) return MORLET_ERR_NOMEM;
  int rc = MORLET_OK;
  const int S = d->n_scales;
  const double wm = d->window_mult > 0 ? d->window_mult : 4.0;
  bool has_adj = false;
  std::vector<FitJob> jobs(S);
  double* d_partial = nullptr;
  const int nblk = 64;
  long long maxL = 0;
  {
    p->desc = *d;
    p->lengths.assign(d->lengths, d->lengths + d->n_signals);
    p->sigmas.assign(d->sigmas, d->sigmas + d->n_scales);
    p->desc.lengths = nullptr;
    p->desc.sigmas = nullptr;
    p->form = (d->form == 1) ? 1 : 2;
    p->elem = d->precision == MORLET_FP64 ? 8 : 4;
    p->spin = d->spin_limit > 0 ? d->spin_limit : DEFAULT_SPIN;
    p->x_off.resize(p->lengths.size());
    long long acc = 0;
    for (size_t i = 0; i < p->lengths.size(); ++i) {
      p->x_off[i] = acc;
      acc += p->lengths[i];
    }
    p->n_in = acc;
    p->n_pl = (acc + 3) / 4 * 4;
    CK(cudaGetDevice(&p->device));
    CK(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device));

    const double Cxi = pow(1.0 + exp(-d->xi * d->xi) - 2.0 * exp(-0.75 * d->xi * d->xi), -0.5);
    const double kxi = exp(-0.5 * d->xi * d->xi);
    for (int s = 0; s < S; ++s) {
      FitJob& J = jobs[s];
      const double sg = p->sigmas[s];
      J.sigma = sg;
      J.xi = d->xi;
      J.omega0 = d->method == MORLET_GAUSS ? 0.0 : d->xi / sg;  // no carrier for the Gaussian
      J.L = (long long)ceil(wm * sg);
      J.amp = d->norm ? Cxi * pow(M_PI, -0.25) / sqrt(sg) : 1.0;
      J.kappa_xi = d->norm ? kxi : 0.0;
      J.method = d->method == MORLET_GAUSS ? 1 : d->method == MORLET_MULTIPLY ? 2 : 0;
      J.deriv = d->deriv;
      J.K = d->K;
      J.fit_tol = d->fit_tol;
      const int kmax_fit = d->K > 0 ? d->K : KMAX;
      if (J.method == 0) {
        J.pc = (long long)floor((d->xi / sg) * (double)J.L / M_PI + 0.5);
        J.ph_lo = (int)std::max<long long>(0, J.pc - kmax_fit);
        J.nh = (int)(J.pc + kmax_fit - J.ph_lo);
      } else {
        J.pc = 0;
        J.ph_lo = 0;
        J.nh = kmax_fit;
      }
      if (J.ph_lo + J.nh > J.L) { rc = MORLET_ERR_ARG; goto fail; }  // harmonics must stay below beta p < pi
      if (J.method == 2) J.deriv = 0;
      if (d->transform == MORLET_ASFT) {
        J.n0 = d->n0 > 0 ? d->n0 : std::max(1, (int)floor(sg / 8.0 + 0.5));
        if (J.n0 > J.L) { rc = MORLET_ERR_ARG; goto fail; }
        J.alpha = (double)J.n0 / (sg * sg);
      } else {
        J.n0 = 0;
        J.alpha = 0.0;
      }
      maxL = std::max(maxL, J.L);
    }
    CK(cudaMalloc(&p->d_jobs, sizeof(FitJob) * S));
    CK(cudaMalloc(&p->d_tabs, sizeof(ScaleTab) * S));
    CK(cudaMemsetAsync(p->d_tabs, 0, sizeof(ScaleTab) * S, st));
    CK(cudaMalloc(&d_partial, sizeof(double) * FIT_STRIDE * nblk * S));
    CK(cudaMemcpyAsync(p->d_jobs, jobs.data(), sizeof(FitJob) * S, cudaMemcpyHostToDevice, st));
    CK(run_fit(p->d_jobs, S, maxL, d_partial, nblk, p->d_tabs, 0, ITEMS, p->form, st));
    p->h_tabs.resize(S);
    CK(cudaMemcpyAsync(p->h_tabs.data(), p->d_tabs, sizeof(ScaleTab) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    p->K_fit = 0;
    for (int s = 0; s < S; ++s) p->K_fit = std::max(p->K_fit, (int)p->h_tabs[s].K);
    p->K_kernel = round_k(std::max(
        d->method == MORLET_MULTIPLY ? 2 * p->K_fit - 1 + (d->norm == 1 ? p->K_fit : 0) : p->K_fit, 2));
    if (p->K_kernel < 0) { rc = MORLET_ERR_UNSUPPORTED; goto fail; }
    for (int s = 0; s < S; ++s)
      if (p->h_tabs[s].p0 + p->K_kernel > jobs[s].L) { rc = MORLET_ERR_ARG; goto fail; }
    CK(run_tables(p->d_tabs, p->d_jobs, S, p->K_kernel, ITEMS, p->form, st));
    if (p->form == 1) {
      std::vector<long long> poff(S + 1, 0);
      for (int s = 0; s < S; ++s) poff[s + 1] = poff[s] + (2 * jobs[s].L) / 1024 + 2 + 1024;
      CK(cudaMalloc(&p->d_phase, sizeof(float2) * poff[S]));
      long long* d_poff = nullptr;
      CK(cudaMalloc(&d_poff, sizeof(long long) * (S + 1)));
      CK(cudaMemcpyAsync(d_poff, poff.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice, st));
      cudaError_t e2 = run_phase_tables(p->d_tabs, p->d_jobs, S, p->d_phase, d_poff, st);
      cudaError_t e3 = cudaStreamSynchronize(st);
      cudaFree(d_poff);
      CK(e2);
      CK(e3);
    }
    CK(cudaMemcpyAsync(p->h_tabs.data(), p->d_tabs, sizeof(ScaleTab) * S, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));

    // adjoint: rotating-form tables of every scale from the same fit (whatever the forward's form),
    // each as two virtual scales, the real plane's (weights cM on Re V, 0) and the imaginary plane's
    // (0, -cL on Im V): gx = sum_s Re W_s(Re gW_s) - Im W_s(Im gW_s)
    has_adj = d->method == MORLET_DIRECT && d->transform == MORLET_SFT &&
              !(d->flags & (MORLET_FLAG_EDGE | MORLET_FLAG_NO_ADJOINT));
    if (has_adj) {
      CK(cudaMalloc(&p->d_tabs_adj, sizeof(ScaleTab) * 2 * S));
      CK(cudaMemcpyAsync(p->d_tabs_adj, p->d_tabs, sizeof(ScaleTab) * S, cudaMemcpyDeviceToDevice, st));
      CK(run_tables(p->d_tabs_adj, p->d_jobs, S, p->K_kernel, ITEMS, 2, st));
      std::vector<ScaleTab> rf(S);
      CK(cudaMemcpyAsync(rf.data(), p->d_tabs_adj, sizeof(ScaleTab) * S, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      p->h_tabs_adj.resize(2 * S);
      for (int s = 0; s < S; ++s) {
        ScaleTab a = rf[s], b = rf[s];
        for (int j = 0; j < KMAX; ++j) {
          a.cL[j] = 0.0;
          a.f_cL[j] = 0.f;
          b.cM[j] = 0.0;
          b.f_cM[j] = 0.f;
          b.cL[j] = -rf[s].cL[j];
          b.f_cL[j] = -rf[s].f_cL[j];
        }
        p->h_tabs_adj[2 * s] = a;
        p->h_tabs_adj[2 * s + 1] = b;
      }
      CK(cudaMemcpyAsync(p->d_tabs_adj, p->h_tabs_adj.data(), sizeof(ScaleTab) * 2 * S, cudaMemcpyHostToDevice, st));
      const size_t planes = p->elem * 2 * (size_t)S * (size_t)p->n_pl;
      CK(cudaMalloc(&p->d_gplanes, planes));
      CK(cudaMalloc(&p->d_wplanes, planes));
      std::vector<int64_t> sd(2 * p->lengths.size());
      for (size_t i = 0; i < p->lengths.size(); ++i) {
        sd[2 * i] = p->x_off[i];
        sd[2 * i + 1] = p->lengths[i];
      }
      CK(cudaMalloc(&p->d_sig_desc, sizeof(int64_t) * sd.size()));
      CK(cudaMemcpyAsync(p->d_sig_desc, sd.data(), sizeof(int64_t) * sd.size(), cudaMemcpyHostToDevice, st));
      CK(cudaStreamSynchronize(st));
    }

    // edge mode: pad every signal by the longest reach of any scale's window (L, plus the ASFT
    // shift n0) so that no stored output sees past the replicated samples
    if (d->flags & MORLET_FLAG_EDGE) {
      long long reach = 0;
      for (int s = 0; s < S; ++s) reach = std::max<long long>(reach, jobs[s].L + jobs[s].n0);
      p->pad = reach;
      p->xp_off.resize(p->lengths.size());
      std::vector<int64_t> desc(3 * p->lengths.size());
      long long at = 0;
      for (size_t i = 0; i < p->lengths.size(); ++i) {
        p->xp_off[i] = at;
        desc[3 * i] = p->x_off[i];
        desc[3 * i + 1] = at;
        desc[3 * i + 2] = p->lengths[i];
        at += p->lengths[i] + 2 * reach;
      }
      p->n_xpad = at;
      CK(cudaMalloc(&p->d_xpad, p->elem * (size_t)at));
      CK(cudaMalloc(&p->d_pad_desc, sizeof(int64_t) * desc.size()));
      CK(cudaMemcpy(p->d_pad_desc, desc.data(), sizeof(int64_t) * desc.size(), cudaMemcpyHostToDevice));
    }
    // work tables and status arrays
    p->ss_min_L = SS_MIN_L;
    p->ls_max_L = LS_MAX_L;
    long long slots = 0;
    rc = setup_launch(p, false, p->fwd, slots);
    if (rc) goto fail;
    long long slots_adj = 0;
    if (has_adj) {
      // The adjoint's rows (compensated FP32) as start-state items for every row, 64 tiles each,
      // longest first: the schedule the autotuner picks for the forward of a large batch
      const long long ss0 = p->ss_min_L, t0 = p->ss_tiles_max;
      const int o0 = p->order;
      if (p->desc.precision == MORLET_FP32_COMP) {
        p->ss_min_L = 1;
        p->ss_tiles_max = 64;
        p->order = 2;
      }
      rc = setup_launch(p, true, p->adj, slots_adj);
      p->ss_min_L = ss0;
      p->ss_tiles_max = t0;
      p->order = o0;
      if (rc) goto fail;
    }
    p->nt_slot = p->K_kernel;
    rc = alloc_slots(p, std::max(slots, slots_adj));
    if (rc) goto fail;
    if (p->fwd.n_pwork > 0) {
      rc = alloc_prefix(p, p->fwd);
      if (rc) goto fail;
    }
    if (p->adj.n_pwork > 0) {
      rc = alloc_prefix(p, p->adj);
      if (rc) goto fail;
    }
    CK(cudaMalloc(&p->d_ticket, sizeof(unsigned long long) * TICKETS * 2));
    CK(cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    CK(cudaHostAlloc((void**)&p->h_err, sizeof(int), cudaHostAllocMapped));
    *p->h_err = 0;
    CK(cudaHostGetDevicePointer((void**)&p->d_err, p->h_err, 0));
    if (d->flags & MORLET_FLAG_AUTOTUNE) {
      rc = autotune(p, st);
      if (rc) goto fail;
    }
  }
  cudaFree(d_partial);
  *out = p;
  return MORLET_OK;
fail:
  cudaFree(d_partial);
  morlet_plan_destroy(p);
  return rc;
}

int morlet_forward(morlet_plan_t p, const void* x, void* W, void* stream) {
  if (!p || !x || !W) return MORLET_ERR_ARG;
  int rc = check_latched(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const bool use_graph = !(p->desc.flags & MORLET_FLAG_NO_GRAPH) && p->skip_tickets == 0;
  if (!use_graph) return cuda_status(forward_enqueue(p, x, W, st));
  const cudaError_t e = forward_graph(p, x, W);
  if (e != cudaSuccess) return cuda_status(e);
  return cuda_status(cudaGraphLaunch(p->gexec, st));
}

int morlet_backward(morlet_plan_t p, const void* gW, void* gx, void* stream) {
  if (!p || !gW || !gx) return MORLET_ERR_ARG;
  if (!p->adj.func) return MORLET_ERR_UNSUPPORTED;
  int rc = check_latched(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const bool use_graph = !(p->desc.flags & MORLET_FLAG_NO_GRAPH) && p->skip_tickets == 0;
  if (!use_graph) return cuda_status(backward_enqueue(p, gW, gx, st));
  const cudaError_t e = capture_graph(p, true, gW, gx);
  if (e != cudaSuccess) return cuda_status(e);
  return cuda_status(cudaGraphLaunch(p->gexec_b, st));
}

int morlet_last_device_error(morlet_plan_t p, void* stream) {
  if (!p) return MORLET_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e);
  int rc = check_latched(p);
  *(volatile int*)p->h_err = 0;
  p->latched = 0;
  return rc;
}

int morlet_plan_info(morlet_plan_t p, int32_t s, int64_t* L, int32_t* p0, int32_t* K, double* m, double* l,
                     int32_t* n0) {
  if (!p || s < 0 || s >= (int32_t)p->h_tabs.size()) return MORLET_ERR_ARG;
  const ScaleTab& t = p->h_tabs[s];
  if (L) *L = t.L;
  if (p0) *p0 = t.p0;
  if (K) *K = t.K;
  if (m) memcpy(m, t.m, sizeof(double) * KMAX);
  if (l) memcpy(l, t.l, sizeof(double) * KMAX);
  if (n0) *n0 = t.n0;
  return MORLET_OK;
}

int morlet_plan_stats(morlet_plan_t p, int64_t o[15]) {
  if (!p || !o) return MORLET_ERR_ARG;
  const Launch& f = p->fwd;
  const bool two = f.func_w != nullptr;
  const long long c_end = two ? f.chain_end : f.n_work;
  const long long s_beg = two ? std::min(std::max(f.ss_begin, c_end), f.n_work) : f.n_work;
  o[0] = THREADS;
  o[1] = ITEMS;
  o[2] = f.grid;
  o[3] = f.n_work;
  o[4] = f.sub_tiles;
  o[5] = f.rows_chain;
  o[6] = f.rows_halo;
  o[7] = (c_end > 0) + (s_beg > c_end) + (f.n_work > s_beg) + (f.n_pwork > 0 && f.n_work > s_beg) + (f.n_lwork > 0);
  o[8] = f.rows_ss;
  o[9] = f.n_pwork;
  o[10] = f.rows_lane;
  o[11] = f.n_lwork;
  o[12] = p->ls_max_L;
  o[13] = p->ss_min_L;
  o[14] = f.ss_window;
  return MORLET_OK;
}

int morlet_plan_set_spin_limit(morlet_plan_t p, int64_t polls) {
  if (!p || polls < 1) return MORLET_ERR_ARG;
  p->spin = polls;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  if (p->gexec_b) {
    cudaGraphExecDestroy(p->gexec_b);
    p->gexec_b = nullptr;
  }
  return MORLET_OK;
}

int morlet_plan_set_row_thresholds(morlet_plan_t p, int64_t lane_chunk_max_L, int64_t start_state_min_L) {
  if (!p || lane_chunk_max_L < 0 || lane_chunk_max_L > LS_MAX_L_MAX || start_state_min_L < 1) return MORLET_ERR_ARG;
  if (p->h_err && *(volatile int*)p->h_err) return MORLET_ERR_TIMEOUT;
  // the ASFT and the multiplication method: Horner start states for the rows with L above the
  // limit (<= 4096)
  if (horner_capable(p)) {
    if (start_state_min_L > TILE) return MORLET_ERR_ARG;
    const long long old_h = p->h_ss_min_L;
    p->h_ss_min_L = start_state_min_L;
    long long slots = 0;
    int rc = build_forward(p, slots);
    if (rc != MORLET_OK) {
      p->h_ss_min_L = old_h;
      long long s2 = 0;
      const int rc2 = build_forward(p, s2);
      return rc2 != MORLET_OK ? rc2 : rc;
    }
    return MORLET_OK;
  }
  if (start_state_min_L > SS_MIN_L_MAX) return MORLET_ERR_ARG;
  const morlet_plan_desc& d = p->desc;
  if (!sft_schedulable(p)) return MORLET_OK;  // a single schedule
  const long long old_ls = p->ls_max_L, old_ss = p->ss_min_L;
  p->ls_max_L = lane_chunk_max_L;
  p->ss_min_L = start_state_min_L;
  long long slots = 0;
  int rc = build_forward(p, slots);
  if (rc != MORLET_OK) {  // back to the thresholds the plan had
    p->ls_max_L = old_ls;
    p->ss_min_L = old_ss;
    long long s2 = 0;
    const int rc2 = build_forward(p, s2);
    return rc2 != MORLET_OK ? rc2 : rc;
  }
  return MORLET_OK;
}

int morlet_plan_set_schedule(morlet_plan_t p, int32_t seg_mult, int32_t ss_tiles_max, int32_t order,
                             int32_t asft_chains) {
  if (!p || (seg_mult != 8 && seg_mult != 12 && seg_mult != 16) || ss_tiles_max < 4 || ss_tiles_max > 64 ||
      order < 0 || order > 2 || asft_chains < 0 || asft_chains > 1)
    return MORLET_ERR_ARG;
  if (p->h_err && *(volatile int*)p->h_err) return MORLET_ERR_TIMEOUT;
  const Sched old = get_sched(p);
  Sched c = old;
  c.seg_mult = seg_mult;
  c.ss_tiles = ss_tiles_max;
  c.order = order;
  c.asft_chains = asft_chains;
  put_sched(p, c);
  long long slots = 0;
  int rc = build_forward(p, slots);
  if (rc != MORLET_OK) {  // back to the schedule the plan had
    put_sched(p, old);
    long long s2 = 0;
    const int rc2 = build_forward(p, s2);
    return rc2 != MORLET_OK ? rc2 : rc;
  }
  return MORLET_OK;
}

int morlet_plan_schedule(morlet_plan_t p, int64_t o[8]) {
  if (!p || !o) return MORLET_ERR_ARG;
  o[0] = p->ls_max_L;
  o[1] = horner_capable(p) ? p->h_ss_min_L : p->ss_min_L;
  o[2] = p->seg_mult;
  o[3] = p->ss_tiles_max;
  o[4] = p->order;
  o[5] = p->asft_chains;
  o[6] = p->tuned;
  o[7] = p->tune_outputs;
  return MORLET_OK;
}

int morlet_debug_skip_tickets(morlet_plan_t p, int64_t skip) {
  if (!p || skip < 0) return MORLET_ERR_ARG;
  p->skip_tickets = skip;
  return MORLET_OK;
}

int gauss_smooth(const void* x, int64_t N, double sigma, int32_t P, int32_t deriv, int32_t precision, void* y,
                 void* stream) {
  if (!x || !y || N < 1 || P < 0 || P + 1 > KMAX || deriv < 0 || deriv > 2) return MORLET_ERR_ARG;
  if (precision < MORLET_FP32_PLAIN || precision > MORLET_FP64) return MORLET_ERR_ARG;
  // Plans are cached per key; the cache lives until process exit.
  static std::mutex mu;
  static std::map<std::tuple<int, int64_t, double, int, int, int>, morlet_plan_t> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MORLET_ERR_CUDA;
  morlet_plan_t plan = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(dev, N, sigma, P, deriv, precision);
    auto it = cache.find(key);
    if (it != cache.end()) {
      plan = it->second;
    } else {
      morlet_plan_desc d{};
      d.n_signals = 1;
      d.lengths = &N;
      d.n_scales = 1;
      d.sigmas = &sigma;
      d.K = P + 1;
      d.method = MORLET_GAUSS;
      d.transform = MORLET_SFT;
      d.precision = precision;
      d.deriv = deriv;
      const int rc = morlet_plan(&plan, &d, stream);
      if (rc) return rc;
      cache[key] = plan;
    }
  }
  return morlet_forward(plan, x, y, stream);
}

}  // extern "C"
