// morlet_forward_noalloc: a forward transform that allocates no memory at all, for callers that
// cannot call cudaMalloc (for example code running under an allocator that forbids it, or inside a
// framework that owns all device memory). Every buffer the transform needs besides the caller's
// input and output lives in one file-scope device array of fixed size, held by each GPU that loads
// this library until the process exits.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "../../include/morlet_sft.h"
#include "plan_internal.h"
#include "work_plan.h"

namespace msft {

namespace {

constexpr int NA_THREADS_ITEMS = 16;
constexpr long long NA_TILE = (long long)THREADS * NA_THREADS_ITEMS;
constexpr long long NA_MAX_ITEMS = 16384;  // work items (sub-tiles) one call may use
constexpr long long NA_MAX_SLOTS = 16384;  // look-back status slots one call may use
constexpr int NA_FIT_BLOCKS = 64;

// Byte layout of the scratch array (every part 256-byte aligned).
constexpr size_t al(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t OFF_TAB = 0;
constexpr size_t OFF_JOB = al(OFF_TAB + sizeof(ScaleTab));
constexpr size_t OFF_PART = al(OFF_JOB + sizeof(FitJob));
constexpr size_t OFF_CHAIN = al(OFF_PART + sizeof(double) * FIT_STRIDE * NA_FIT_BLOCKS);
constexpr size_t OFF_WORK = al(OFF_CHAIN + sizeof(ChainDesc));
constexpr size_t OFF_FLAGS = al(OFF_WORK + sizeof(WorkItem) * NA_MAX_ITEMS);
constexpr size_t OFF_AGG = al(OFF_FLAGS + sizeof(uint32_t) * NA_MAX_SLOTS);
constexpr size_t OFF_INCL = al(OFF_AGG + sizeof(double2) * KMAX * NA_MAX_SLOTS);
constexpr size_t OFF_TICKET = al(OFF_INCL + sizeof(double2) * KMAX * NA_MAX_SLOTS);
constexpr size_t OFF_ERR = al(OFF_TICKET + sizeof(unsigned long long));
constexpr size_t NA_SCRATCH_BYTES = al(OFF_ERR + sizeof(int));

// The scratch array. In host code `na_scratch` is only a stand-in symbol, not a device address:
// the address every kernel receives comes from cudaGetSymbolAddress, taken once per device.
static __device__ __align__(256) unsigned char na_scratch[NA_SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mu;
unsigned char* na_addr[NA_MAX_DEVICES] = {nullptr};
// The row's work items are cut on the host (the same decomposition as the plan's, work_plan.h) into
// this file-scope host array and copied into the scratch array with one copy; guarded by na_mu.
WorkItem na_items[NA_MAX_ITEMS];

int na_status(cudaError_t e) {
  if (e == cudaSuccess) return MORLET_OK;
  if (e == cudaErrorMemoryAllocation) return MORLET_ERR_NOMEM;
  return MORLET_ERR_CUDA;
}

}  // namespace
}  // namespace msft

using namespace msft;

extern "C" int morlet_forward_noalloc(const void* x, int64_t N, double sigma, double xi, int32_t K, void* W,
                                      void* stream) {
  if (!x || !W || N < 1 || !(sigma >= 0.5) || !(sigma < 1e9) || !(xi >= 0.0 && xi < 1e6)) return MORLET_ERR_ARG;
  if (K < 1 || K > KMAX) return MORLET_ERR_ARG;
  int kk = -1;
  for (int i = 0; i < N_KBUILT; ++i)
    if (kbuilt(i) >= std::max(K, 2)) {
      kk = kbuilt(i);
      break;
    }
  if (kk < 0) return MORLET_ERR_UNSUPPORTED;
  const long long L = (long long)ceil(4.0 * sigma);
  const long long pc = (long long)floor((xi / sigma) * (double)L / M_PI + 0.5);
  const long long ph_lo = std::max<long long>(0, pc - K);
  if (pc + kk > L) return MORLET_ERR_ARG;  // every harmonic p0 + j must stay below L (beta p < pi)
  // the row as the plan describes it (32-byte aligned segment starts, window segments on the warp
  // kernel); size limits of the scratch array
  const RowSpec r = make_row_spec(N, L, L, 0, 0, 0, (int)sizeof(float), SEG_RESTART, 0, true, NA_TILE, 0, 0, 16);
  long long n_slots = 0, n_sub = 0;
  bool chained = false;
  const long long n_work = row_work(r, NA_TILE, nullptr, &n_slots, &n_sub, &chained);
  if (n_work > NA_MAX_ITEMS || n_slots > NA_MAX_SLOTS) return MORLET_ERR_ARG;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_status(e);
  if (dev < 0 || dev >= NA_MAX_DEVICES) return MORLET_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(na_mu);  // the host item array and the set-up below
  if (!na_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, na_scratch);  // device address of the array on this device
    if (e != cudaSuccess || !ptr) return na_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    na_addr[dev] = (unsigned char*)ptr;
  }
  unsigned char* const base = na_addr[dev];
  cudaStream_t st = (cudaStream_t)stream;

  // a timeout latched by the previous call on this device is reported now
  int prev_err = 0;
  e = cudaMemcpyAsync(&prev_err, base + OFF_ERR, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_status(e);

  FitJob J{};
  J.sigma = sigma;
  J.xi = xi;
  J.omega0 = xi / sigma;
  J.L = L;
  J.amp = 1.0;
  J.kappa_xi = 0.0;
  J.method = 0;
  J.K = K;
  J.pc = pc;
  J.ph_lo = (int)ph_lo;
  J.nh = (int)(pc + K - ph_lo);
  J.n0 = 0;
  J.alpha = 0.0;
  FitJob* d_job = (FitJob*)(base + OFF_JOB);
  ScaleTab* d_tab = (ScaleTab*)(base + OFF_TAB);
  e = cudaMemcpyAsync(d_job, &J, sizeof(FitJob), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_tab, 0, sizeof(ScaleTab), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + OFF_ERR, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = run_fit(d_job, 1, L, (double*)(base + OFF_PART), NA_FIT_BLOCKS, d_tab, kk, NA_THREADS_ITEMS, 2, st);
  if (e == cudaSuccess) e = run_tables(d_tab, d_job, 1, kk, NA_THREADS_ITEMS, 2, st);
  ChainDesc* d_chain = (ChainDesc*)(base + OFF_CHAIN);
  WorkItem* d_work = (WorkItem*)(base + OFF_WORK);
  ChainDesc chain{};
  chain.n = N;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_chain, &chain, sizeof(ChainDesc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    // host memory that is not page-locked: each copy returns once its source has been read, so the
    // host array and the stack values above may be reused right after
    long long s2 = 0, t2 = 0;
    bool c2 = false;
    row_work(r, NA_TILE, na_items, &s2, &t2, &c2);
    e = cudaMemcpyAsync(d_work, na_items, sizeof(WorkItem) * (size_t)n_work, cudaMemcpyHostToDevice, st);
  }
  // the counter and the status flags must start at zero for every call
  if (e == cudaSuccess) e = cudaMemsetAsync(base + OFF_TICKET, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess && n_slots > 0) e = cudaMemsetAsync(base + OFF_FLAGS, 0, sizeof(uint32_t) * n_slots, st);
  if (e != cudaSuccess) return na_status(e);

  // look-back rows on the CTA kernel, window rows on the warp-independent kernel (as the plan does)
  const void* func = kernel_for(V_RF_F32C_MORLET, kk, !chained);
  if (!func) return MORLET_ERR_UNSUPPORTED;
  int sms = 0, occ = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, func, THREADS, 0);
  if (e != cudaSuccess) return na_status(e);
  KParams kp{};
  kp.x = x;
  kp.out = W;
  kp.work = d_work;
  kp.n_work = n_work;
  kp.chains = d_chain;
  kp.tabs = d_tab;
  kp.flags = (uint32_t*)(base + OFF_FLAGS);
  kp.agg = base + OFF_AGG;
  kp.incl = base + OFF_INCL;
  kp.ticket = (unsigned long long*)(base + OFF_TICKET);
  kp.err = (int*)(base + OFF_ERR);
  kp.spin_limit = 1LL << 20;
  kp.n_chain = chained ? n_work : 0;
  kp.n_x = N;
  void* args[] = {&kp};
  const long long units = chained ? n_work : (n_work + WARPS - 1) / WARPS;  // CTAs, or warps per CTA
  const int grid = (int)std::min<long long>((long long)std::max(occ, 1) * sms, units);
  e = cudaLaunchKernel(func, dim3(grid), dim3(THREADS), args, 0, st);
  if (e != cudaSuccess) return na_status(e);
  return prev_err ? MORLET_ERR_TIMEOUT : MORLET_OK;
}
