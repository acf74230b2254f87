// Flux kernel instantiations: working precision float, direction 1.
#define HX_FLUX_R float
#define HX_FLUX_NAME f32_d
#define HX_FLUX_DIR 1
#include "k_flux_inst.cuh"
