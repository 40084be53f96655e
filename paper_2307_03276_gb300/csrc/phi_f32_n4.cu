// Phi / MTTKRP / log-likelihood tile kernels: float, 5-way tensors.
#define PHI_T float
#define PHI_IS_DOUBLE 0
#define PHI_NM1 4
#define PHI_FN launch_phi_f32_n4
#include "phi_inst.cuh"
