// Prefix-sum and tile-sum kernel instantiations (compensated FP32, real input):
// `const void* kernel_psum(int K)`, `const void* kernel_tsum(int K)`.
#include "kernels_inst.cuh"

namespace msft {
const void* kernel_psum(int K) {
  switch (K) {
    case 2: return (const void*)&psum_kernel<Cfg<float, DFC, 2, FORM_RF, OUT_MORLET, false, 16>>;
    case 3: return (const void*)&psum_kernel<Cfg<float, DFC, 3, FORM_RF, OUT_MORLET, false, 16>>;
    case 4: return (const void*)&psum_kernel<Cfg<float, DFC, 4, FORM_RF, OUT_MORLET, false, 16>>;
    case 6: return (const void*)&psum_kernel<Cfg<float, DFC, 6, FORM_RF, OUT_MORLET, false, 16>>;
    case 8: return (const void*)&psum_kernel<Cfg<float, DFC, 8, FORM_RF, OUT_MORLET, false, 16>>;
    case 12: return (const void*)&psum_kernel<Cfg<float, DFC, 12, FORM_RF, OUT_MORLET, false, 16>>;
    default: return nullptr;
  }
}
}  // namespace msft

namespace msft {
const void* kernel_tsum(int K) {
  switch (K) {
    case 2: return (const void*)&tsum_kernel<Cfg<float, DFC, 2, FORM_RF, OUT_MORLET, false, 16>>;
    case 3: return (const void*)&tsum_kernel<Cfg<float, DFC, 3, FORM_RF, OUT_MORLET, false, 16>>;
    case 4: return (const void*)&tsum_kernel<Cfg<float, DFC, 4, FORM_RF, OUT_MORLET, false, 16>>;
    case 6: return (const void*)&tsum_kernel<Cfg<float, DFC, 6, FORM_RF, OUT_MORLET, false, 16>>;
    case 8: return (const void*)&tsum_kernel<Cfg<float, DFC, 8, FORM_RF, OUT_MORLET, false, 16>>;
    case 12: return (const void*)&tsum_kernel<Cfg<float, DFC, 12, FORM_RF, OUT_MORLET, false, 16>>;
    default: return nullptr;
  }
}
}  // namespace msft

namespace msft {
// Horner tile sums (the ASFT's damped rho, the multiplication method's non-harmonic rho); the kernel
// reads only K, ITEMS and the Horner switch of its configuration, so one instance serves both
const void* kernel_tsum_h(int K) {
  switch (K) {
    case 2: return (const void*)&tsum_kernel<Cfg<float, float2, 2, FORM_RF, OUT_MORLET, true, 16>>;
    case 3: return (const void*)&tsum_kernel<Cfg<float, float2, 3, FORM_RF, OUT_MORLET, true, 16>>;
    case 4: return (const void*)&tsum_kernel<Cfg<float, float2, 4, FORM_RF, OUT_MORLET, true, 16>>;
    case 6: return (const void*)&tsum_kernel<Cfg<float, float2, 6, FORM_RF, OUT_MORLET, true, 16>>;
    case 8: return (const void*)&tsum_kernel<Cfg<float, float2, 8, FORM_RF, OUT_MORLET, true, 16>>;
    case 12: return (const void*)&tsum_kernel<Cfg<float, float2, 12, FORM_RF, OUT_MORLET, true, 16>>;
    default: return nullptr;
  }
}
}  // namespace msft
