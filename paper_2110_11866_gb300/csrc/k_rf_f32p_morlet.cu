// Scan kernel instantiations: rf f32p morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_morlet, float, float, FORM_RF, OUT_MORLET, false, 16)
