// The FP32 stage kernel's launcher for the primitive-departure reconstruction (gamma = 7/5 powers).
#define ROSSBI_RC RECON_PRIM
#include "k_stage_pert_f32.cu"
