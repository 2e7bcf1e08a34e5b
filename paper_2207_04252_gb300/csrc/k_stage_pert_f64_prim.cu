// The FP64 perturbation-form stage kernel's launcher for the primitive-departure reconstruction.
#define ROSSBI_RC RECON_PRIM
#include "k_stage_pert_f64.cu"
