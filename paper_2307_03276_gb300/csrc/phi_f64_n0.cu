// Phi / MTTKRP / log-likelihood tile kernels: double, any number of modes (runtime count).
#define PHI_T double
#define PHI_IS_DOUBLE 1
#define PHI_NM1 0
#define PHI_FN launch_phi_f64_n0
#include "phi_inst.cuh"
