// The FP64 stage kernel's launcher for the primitive-departure reconstruction.
#define ROSSBI_RC RECON_PRIM
#include "k_stage_full.cu"
