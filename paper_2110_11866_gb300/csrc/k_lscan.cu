// Lane-chunk scan instantiations (compensated FP32 SFT Morlet): `const void* kernel_lscan(int K)`.
#include "kernels_inst.cuh"
#include "lscan_kernel.cuh"

namespace msft {
const void* kernel_lscan(int K) {
  switch (K) {
    case 2: return (const void*)&lscan_kernel<Cfg<float, DFC, 2, FORM_RF, OUT_MORLET, false, 16>>;
    case 3: return (const void*)&lscan_kernel<Cfg<float, DFC, 3, FORM_RF, OUT_MORLET, false, 16>>;
    case 4: return (const void*)&lscan_kernel<Cfg<float, DFC, 4, FORM_RF, OUT_MORLET, false, 16>>;
    case 6: return (const void*)&lscan_kernel<Cfg<float, DFC, 6, FORM_RF, OUT_MORLET, false, 16>>;
    case 8: return (const void*)&lscan_kernel<Cfg<float, DFC, 8, FORM_RF, OUT_MORLET, false, 16>>;
    case 12: return (const void*)&lscan_kernel<Cfg<float, DFC, 12, FORM_RF, OUT_MORLET, false, 16>>;
    default: return nullptr;
  }
}
}  // namespace msft
