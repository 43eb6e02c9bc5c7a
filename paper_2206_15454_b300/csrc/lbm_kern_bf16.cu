// lbm_kern_bf16.cu -- the kernels of one storage type (see lbm_kern.inc).
#define LBM_KERN_S 2
#include "lbm_kern.inc"
