// Internal declarations shared by the plan (host) and the plan-time GPU kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace msft {

// One scale's fit problem (filled on the host, read by the FP64 fit kernels).
struct FitJob {
  double sigma, xi, omega0;
  double amp;        // Morlet amplitude (1, or C_xi pi^{-1/4} sigma^{-1/2} for norm = 1)
  double kappa_xi;   // Morlet offset (0, or kappa_xi for norm = 1)
  double alpha;      // ASFT decay (0 for SFT)
  double fit_tol;    // automatic K
  long long L;       // half window
  long long pc;      // harmonic nearest the carrier, floor(omega0 L / pi + 1/2)
  int32_t ph_lo, nh; // harmonics [ph_lo, ph_lo + nh) whose right-hand sides are summed
  int32_t method;    // 0 Morlet direct, 1 Gaussian
  int32_t deriv;
  int32_t K;         // 0 = automatic
  int32_t n0;        // ASFT shift (0 for SFT)
};

constexpr int FIT_STRIDE = 4 * KMAX + 1;

cudaError_t run_fit(const FitJob* d_jobs, int n_scales, long long max_L, double* d_partial, int nblk,
                    ScaleTab* d_tabs, int K_kernel, int items, int form, cudaStream_t st);
cudaError_t run_tables(ScaleTab* d_tabs, const FitJob* d_jobs, int n_scales, int K_kernel, int items, int form,
                       cudaStream_t st);

cudaError_t run_phase_tables(ScaleTab* d_tabs, const FitJob* d_jobs, int n_scales, float2* d_phase,
                             const long long* d_poff, cudaStream_t st);

// Kernel lookup: the scan kernel of a variant and a built term count, or nullptr.
enum Variant {
  V_RF_F32C_MORLET = 0,  // rotating form, FP32 scan, two-float carries
  V_RF_F32P_MORLET,      // rotating form, FP32 scan, FP32 carries
  V_RF_F32P_ASFT,        // ASFT, FP32
  V_RF_F64_MORLET,
  V_KI_F32C_MORLET,      // kernel-integral form
  V_KI_F32P_MORLET,
  V_KI_F64_MORLET,
  V_RF_F32C_REAL,        // Gaussian smoothing
  V_RF_F32P_REAL,
  V_RF_F64_REAL,
  V_RF_F32P_ASFT_REAL,   // ASFT Gaussian smoothing, FP32
  V_RF_F32P_MULT,        // multiplication method, FP32
  V_COUNT
};

// K values that have a compiled kernel; a plan rounds its K up to the next one.
constexpr int N_KBUILT = 6;
__host__ __device__ constexpr int kbuilt(int i) { return i == 0 ? 2 : i == 1 ? 3 : i == 2 ? 4 : i == 3 ? 6 : i == 4 ? 8 : 12; }

const void* kernel_for(int variant, int K, bool warp);
const void* kernel_psum(int K);   // prefix sums of the start-state rows (k_psum.cu)
const void* kernel_tsum(int K);   // tile sums of the start-state rows (k_psum.cu)
const void* kernel_tsum_h(int K); // Horner tile sums: ASFT and multiplication-method start-state rows
const void* kernel_lscan(int K);  // lane-chunk scan of short-window rows (k_lscan.cu)

}  // namespace msft
