// Scan kernel instantiations: ki f64 morlet.
#include "kernels_inst.cuh"
MSFT_INST(kernel_ki_f64_morlet, double, double2, FORM_KI, OUT_MORLET, false, 16)
