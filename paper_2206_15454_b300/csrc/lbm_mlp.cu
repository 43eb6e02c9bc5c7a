// lbm_mlp.cu -- launchers of the correction network's kernels (lbm_mlp.cuh),
// compiled in a translation unit of their own.
#include "lbm_kernels.h"
#include "lbm_mlp.cuh"

namespace lbm {

void mlp_launch_infer(int blocks, cudaStream_t s, const float* th, const float* X, long long n,
                      float* Y) {
  mlp_infer_kernel<<<blocks, 128, 0, s>>>(th, X, n, Y);
}

void mlp_launch_train_fwd(int blocks, cudaStream_t s, const float* th, const float* X,
                          const float* Y, const int* idx, int n, float scale, float* H0, float* H1,
                          float* H2, float* H3, float* D4, float* sse) {
  mlp_train_fwd<<<blocks, 128, 0, s>>>(th, X, Y, idx, n, scale, H0, H1, H2, H3, D4, sse);
}

void mlp_launch_train_bwd(int blocks, cudaStream_t s, const float* th, int n, const float* H1,
                          const float* H2, const float* H3, const float* D4, float* D1, float* D2,
                          float* D3) {
  mlp_train_bwd<<<blocks, 128, 0, s>>>(th, n, H1, H2, H3, D4, D1, D2, D3);
}

void mlp_launch_train_wgrad(dim3 grid, cudaStream_t s, const float* D, int nout, const float* Hin,
                            int nin, int n, int rows_per_slice, float* gW, float* gb) {
  mlp_train_wgrad<<<grid, 256, 0, s>>>(D, nout, Hin, nin, n, rows_per_slice, gW, gb);
}

void mlp_launch_adam(int blocks, cudaStream_t s, float* th, const float* g, float* m, float* v,
                     int n, float lr, float c1, float c2) {
  mlp_adam<<<blocks, 256, 0, s>>>(th, g, m, v, n, lr, c1, c2);
}

}  // namespace lbm
