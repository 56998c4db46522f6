// Scan kernel instantiations: rf f32p real.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_real, float, float, FORM_RF, OUT_REAL, false, 16)
