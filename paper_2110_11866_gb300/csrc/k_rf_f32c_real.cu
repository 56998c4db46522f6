// Scan kernel instantiations: rf f32c real.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32c_real, float, double, FORM_RF, OUT_REAL, false, 16)
