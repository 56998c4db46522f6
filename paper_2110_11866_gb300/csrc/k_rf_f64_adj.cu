// Scan kernel instantiations: rf f64 adj.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f64_adj, double, double, FORM_RF, OUT_ADJ, false, 16)
