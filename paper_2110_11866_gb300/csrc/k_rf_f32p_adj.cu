// Scan kernel instantiations: rf f32p adj.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_adj, float, float, FORM_RF, OUT_ADJ, false, 16)
