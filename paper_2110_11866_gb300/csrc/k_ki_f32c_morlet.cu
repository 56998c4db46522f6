// Scan kernel instantiations: ki f32c morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_ki_f32c_morlet, float, DFC, FORM_KI, OUT_MORLET, false, 16)
