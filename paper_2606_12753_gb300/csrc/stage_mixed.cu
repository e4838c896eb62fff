// Stage-kernel instantiations and launchers for the mixed form.
#define MHD_UNIT_PREC P_MIXED
#define MHD_UNIT_FN(name) name##_mixed
#define MHD_TILES(X) X(16, 8) X(16, 16) X(32, 8) X(24, 8) X(8, 8)
#include "stage_unit.cuh"
