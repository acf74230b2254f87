// Flux kernel instantiations: working precision double, direction 1.
#define HX_FLUX_R double
#define HX_FLUX_NAME f64_d
#define HX_FLUX_DIR 1
#include "k_flux_inst.cuh"
