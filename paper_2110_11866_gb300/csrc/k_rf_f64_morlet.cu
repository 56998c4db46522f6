// Scan kernel instantiations: rf f64 morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f64_morlet, double, double, FORM_RF, OUT_MORLET, false, 16)
