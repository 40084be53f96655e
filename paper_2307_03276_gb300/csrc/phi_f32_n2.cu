// Phi / MTTKRP / log-likelihood tile kernels: float, 3-way tensors.
#define PHI_T float
#define PHI_IS_DOUBLE 0
#define PHI_NM1 2
#define PHI_FN launch_phi_f32_n2
#include "phi_inst.cuh"
