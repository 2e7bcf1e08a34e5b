// The FP32 stage kernel's launcher for a general gamma (log1p / expm1 powers).
#define ROSSBI_POW PowGeneric<float>
#include "k_stage_pert_f32.cu"
