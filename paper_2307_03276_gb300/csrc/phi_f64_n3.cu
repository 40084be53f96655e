// Phi / MTTKRP / log-likelihood tile kernels: double, 4-way tensors.
#define PHI_T double
#define PHI_IS_DOUBLE 1
#define PHI_NM1 3
#define PHI_FN launch_phi_f64_n3
#include "phi_inst.cuh"
