// Scan kernel instantiations: rf f64 real.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f64_real, double, double, FORM_RF, OUT_REAL, false, 16)
