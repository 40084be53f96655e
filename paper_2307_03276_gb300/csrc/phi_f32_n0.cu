// Phi / MTTKRP / log-likelihood tile kernels: float, any number of modes (runtime count).
#define PHI_T float
#define PHI_IS_DOUBLE 0
#define PHI_NM1 0
#define PHI_FN launch_phi_f32_n0
#include "phi_inst.cuh"
