// Plain FP64 path: every quantity in double precision.
#define REED_R double
#define REED_NS reed_f64
#include "reed_kernels.inc"
