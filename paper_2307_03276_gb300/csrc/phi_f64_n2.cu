// Phi / MTTKRP / log-likelihood tile kernels: double, 3-way tensors.
#define PHI_T double
#define PHI_IS_DOUBLE 1
#define PHI_NM1 2
#define PHI_FN launch_phi_f64_n2
#include "phi_inst.cuh"
