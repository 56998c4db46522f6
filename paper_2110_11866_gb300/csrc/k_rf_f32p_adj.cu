// Scan kernel instantiations: rf f32p adj.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_adj, float, float2, FORM_RF, OUT_ADJ, false, 16)
MSFT_INST_W(kernel_rf_f32p_adj_w, float, float2, OUT_ADJ, false, 16)
