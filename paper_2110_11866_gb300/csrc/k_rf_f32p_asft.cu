// Scan kernel instantiations: rf f32p asft.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_asft, float, float, FORM_RF, OUT_MORLET, true, 16)
