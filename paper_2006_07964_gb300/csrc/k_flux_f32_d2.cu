// Flux kernel instantiations: working precision float, direction 2.
#define HX_FLUX_R float
#define HX_FLUX_NAME f32_d
#define HX_FLUX_DIR 2
#include "k_flux_inst.cuh"
