// Scan kernel instantiations: rf f32p mult (multiplication method: non-harmonic terms, complex combine).
#include "kernels_inst.cuh"
MSFT_INST(kernel_rf_f32p_mult, float, float2, FORM_RF, OUT_CPLX, true, 16)
MSFT_INST_W(kernel_rf_f32p_mult_w, float, float2, OUT_CPLX, true, 16)
