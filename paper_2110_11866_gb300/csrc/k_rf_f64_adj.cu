// Scan kernel instantiations: rf f64 adj.
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f64_adj, double, double2, FORM_RF, OUT_ADJ, false, 16)
MSFT_INST_W(kernel_rf_f64_adj_w, double, double2, OUT_ADJ, false, 16)
