// Scan kernel instantiations: rf f32c morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32c_morlet, float, DFC, FORM_RF, OUT_MORLET, false, 16)
MSFT_INST_W(kernel_rf_f32c_morlet_w, float, DFC, OUT_MORLET, false, 16)
