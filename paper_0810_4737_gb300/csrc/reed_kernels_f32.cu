// Mixed-precision form: FP32 atoms and forces, FP64 ion, time and tallies.
#define REED_R float
#define REED_NS reed_f32
#include "reed_kernels.inc"
