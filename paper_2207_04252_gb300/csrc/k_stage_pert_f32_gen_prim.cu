// The FP32 stage kernel's launcher for a general gamma and the primitive-departure reconstruction.
#define ROSSBI_RC RECON_PRIM
#define ROSSBI_POW PowGeneric<float>
#include "k_stage_pert_f32.cu"
