// Scan kernel instantiations: rf f64 real.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f64_real, double, double2, FORM_RF, OUT_REAL, false, 16)
MSFT_INST_W(kernel_rf_f64_real_w, double, double2, OUT_REAL, false, 16)
