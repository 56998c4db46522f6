// Scan kernel instantiations: ki f32p morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_ki_f32p_morlet, float, float2, FORM_KI, OUT_MORLET, false, 16)
