// Scan kernel instantiations: rf f32c adj.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32c_adj, float, DFC, FORM_RF, OUT_ADJ, false, 16)
MSFT_INST_W(kernel_rf_f32c_adj_w, float, DFC, OUT_ADJ, false, 16)
