// lbm_kern_f32.cu -- the kernels of one storage type (see lbm_kern.inc).
#define LBM_KERN_S 0
#include "lbm_kern.inc"
