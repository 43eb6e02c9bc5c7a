// lbm_kernels.h -- host-side launchers of the per-(chunk width, storage)
// kernels of lbm_device.cuh and lbm_mlp.cuh.
//
// Every kernel template is instantiated in one of three translation units
// (lbm_kern_f32.cu, lbm_kern_f16.cu, lbm_kern_bf16.cu, one per storage type)
// so the library compiles in parallel; the host code in lbm_api.cu only calls
// these launchers.  All launches are asynchronous on the given stream; launch
// errors surface through cudaGetLastError.
#pragma once

#include <cuda_runtime.h>

#include "lbm_aa.cuh"
#include "lbm_features.cuh"

namespace lbm {

template <int XT, int S>
struct Kern {
  // Largest dynamic shared memory the step kernels may use (stage ring) in
  // the default and in the variant form.
  static void configure(size_t smem_default, size_t smem_variant);
  // Cells per thread along x of the step kernel of that form (1 or 2); its
  // block is (XT / cpt) x (256 cpt / XT) threads.
  static int cells_per_thread(bool variant);
  // Resident blocks per SM of the step kernels of that form.
  static int occupancy(dim3 block, size_t smem, bool variant);
  // One time step (programmatic dependent launch when pdl).  variant: the
  // model-variant form (streamwise-only drag, exact-difference forcing,
  // tau_total with 1/rho^2), selected by the flags in p.
  static void step(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const StepParams& p,
                   bool stats, bool variant, bool pdl);
  // One step of the AA-pattern layout (p.aa_parity: 0 step B, 1 step A) with
  // the tile pipeline of the pull scheme (default model): shared memory,
  // resident blocks per SM and the launch (a programmatic dependent).
  static void aa_configure(size_t smem);
  static int aa_occupancy(dim3 block, size_t smem);
  static void aa_step(dim3 grid, dim3 block, size_t smem, cudaStream_t s, const StepParams& p,
                      bool stats);
  // One time step of every box of an ensemble (work list w).
  static void batch_step(int nblocks, dim3 block, size_t smem, cudaStream_t s,
                         const StepParams* boxes, const BatchWork* w, bool stats);
  static void ghosts(int blocks, cudaStream_t s, const StepParams& p, void* f);
  static void init(int blocks, cudaStream_t s, const InitParams& ip);
  static void mass(int blocks, cudaStream_t s, const void* f, int nx, long long rows, int nxc,
                   double* partial);
  static void macro(int blocks, cudaStream_t s, const StepParams& p, float* out);
  static void macro_d(int blocks, cudaStream_t s, const StepParams& p, double* out);
  static void features(int blocks, cudaStream_t s, const StepParams& p, float* X);
  // The learned correction after a step: column features and network in one
  // pass, the layer-0 acceleration into accel.
  static void correction(int blocks, cudaStream_t s, const StepParams& p, const float* th,
                         float lam, float2* accel);
  static int correction_occupancy();
  // x-halo faces of a slab: pack from / unpack into population set f.
  static void halo_pack(int blocks, cudaStream_t s, const StepParams& p, const void* f, void* lo,
                        void* hi);
  static void halo_unpack(int blocks, cudaStream_t s, const StepParams& p, void* f, const void* lo,
                          const void* hi);
};

// AA-pattern storage (lbm_aa.cuh), per storage type (no chunk width): the
// boundary fill, and the one-cell step of the model-variant form.
template <int S>
struct KernAA {
  static int occupancy();  // resident blocks per SM of the step kernel (256 threads)
  static void fill(cudaStream_t s, const StepParams& p);  // grid: aa_fill_grid
  static void step(int blocks, cudaStream_t s, const AAStep& a, bool stats, bool variant);
  static void init(int blocks, cudaStream_t s, const StepParams& p, const InitParams& ip);
  static void mass(int blocks, cudaStream_t s, const StepParams& p, double* partial);
  static void macro(int blocks, cudaStream_t s, const StepParams& p, float* out);
  static void macro_d(int blocks, cudaStream_t s, const StepParams& p, double* out);
};

// ---- the learned correction's network (lbm_mlp.cu; kernels in lbm_mlp.cuh) ----
void mlp_launch_infer(int blocks, cudaStream_t s, const float* th, const float* X, long long n,
                      float* Y);
void mlp_launch_train_fwd(int blocks, cudaStream_t s, const float* th, const float* X,
                          const float* Y, const int* idx, int n, float scale, float* H0, float* H1,
                          float* H2, float* H3, float* D4, float* sse);
void mlp_launch_train_bwd(int blocks, cudaStream_t s, const float* th, int n, const float* H1,
                          const float* H2, const float* H3, const float* D4, float* D1, float* D2,
                          float* D3);
void mlp_launch_train_wgrad(dim3 grid, cudaStream_t s, const float* D, int nout, const float* Hin,
                            int nin, int n, int rows_per_slice, float* gW, float* gb);
void mlp_launch_adam(int blocks, cudaStream_t s, float* th, const float* g, float* m, float* v,
                     int n, float lr, float c1, float c2);

#define LBM_DECLARE_KERN(SV)           \
  extern template struct Kern<64, SV>; \
  extern template struct Kern<128, SV>; \
  extern template struct Kern<256, SV>;
LBM_DECLARE_KERN(0)
LBM_DECLARE_KERN(1)
LBM_DECLARE_KERN(2)
extern template struct KernAA<0>;
extern template struct KernAA<1>;
extern template struct KernAA<2>;
#undef LBM_DECLARE_KERN

}  // namespace lbm
