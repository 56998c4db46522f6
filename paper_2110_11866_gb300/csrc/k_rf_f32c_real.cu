// Scan kernel instantiations: rf f32c real.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32c_real, float, DFC, FORM_RF, OUT_REAL, false, 16)
MSFT_INST_W(kernel_rf_f32c_real_w, float, DFC, OUT_REAL, false, 16)
