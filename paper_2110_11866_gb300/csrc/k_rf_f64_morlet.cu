// Scan kernel instantiations: rf f64 morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f64_morlet, double, double2, FORM_RF, OUT_MORLET, false, 16)
MSFT_INST_W(kernel_rf_f64_morlet_w, double, double2, OUT_MORLET, false, 16)
