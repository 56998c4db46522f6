// Scan kernel instantiations: rf f32c adj.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32c_adj, float, double, FORM_RF, OUT_ADJ, false, 16)
