// Scan kernel instantiations: rf f32p asft (Morlet output, and real output for Gaussian smoothing).
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_asft, float, float2, FORM_RF, OUT_MORLET, true, 16)
MSFT_INST_W(kernel_rf_f32p_asft_w, float, float2, OUT_MORLET, true, 16)
MSFT_INST(kernel_rf_f32p_asft_real, float, float2, FORM_RF, OUT_REAL, true, 16)
MSFT_INST_W(kernel_rf_f32p_asft_real_w, float, float2, OUT_REAL, true, 16)
