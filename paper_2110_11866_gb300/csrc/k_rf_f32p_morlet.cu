// Scan kernel instantiations: rf f32p morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_morlet, float, float2, FORM_RF, OUT_MORLET, false, 16)
MSFT_INST_W(kernel_rf_f32p_morlet_w, float, float2, OUT_MORLET, false, 16)
