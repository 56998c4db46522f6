// Scan kernel instantiations: rf f32c morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32c_morlet, float, double, FORM_RF, OUT_MORLET, false, 16)
