// lbm_kern_f16.cu -- the kernels of one storage type (see lbm_kern.inc).
#define LBM_KERN_S 1
#include "lbm_kern.inc"
