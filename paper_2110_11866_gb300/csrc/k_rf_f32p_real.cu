// Scan kernel instantiations: rf f32p real.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_real, float, float2, FORM_RF, OUT_REAL, false, 16)
MSFT_INST_W(kernel_rf_f32p_real_w, float, float2, OUT_REAL, false, 16)
