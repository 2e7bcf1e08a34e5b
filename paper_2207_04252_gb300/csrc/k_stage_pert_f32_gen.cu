// Launcher of the FP32 perturbation-form stage kernel (stage_pert.cuh) for a
// general gamma (log1p / expm1 powers); a translation unit of its own so that
// the two float families compile in parallel.
#define ROSSBI_F32_GENERIC_GAMMA
#include "k_stage_pert_f32.cu"
