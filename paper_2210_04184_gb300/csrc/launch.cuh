// Host-side launchers of the kernel families with many template instantiations.  Each family
// is instantiated in its own translation unit (launch_latent.cu, launch_pixel.cu,
// launch_grad.cu, launch_fft.cu), so the library's device code compiles in parallel; the launch sequence in
// fuse_api.cu calls these functions.  Every launcher issues one kernel launch on stream `s`
// and returns without checking it (the caller reads cudaGetLastError).
// Instantiated for T = float with WT = float or __nv_bfloat16, and T = double with WT = double.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "k_grad.cuh"
#include "k_latent.cuh"
#include "k_pixel.cuh"
#include "k_stencil.cuh"
#include "k_wfft.cuh"

namespace fuse {

// ---- latent pass (k_latent.cuh) ----
// Bulk-copy latent pass of one problem; K = patch half-size; int16_state: 16-bit fixed-point
// state (T = float only).
template <typename T, typename WT>
void latent_tma_launch(const LatentArgs<T, WT>& a, int K, bool int16_state, dim3 grid, unsigned threads,
                       size_t smem, cudaStream_t s);
// Batched bulk-copy latent pass over the segment table.
template <typename T, typename WT>
void latent_tma_batch_launch(const LatentArgs<T, WT>* args, const Segment* seg, int nseg, int zero_in, int K,
                             bool int16_state, unsigned blocks, unsigned threads, size_t smem, cudaStream_t s);
// Register-staged latent pass.
template <typename T, typename WT>
void latent_reg_launch(const T* X, const WT* omega, const T* Sig, T* Sout, T* planes, int H, int W, int Ls, int S,
                       int Ty, T coef, int half, int K, dim3 grid, unsigned threads, size_t smem, cudaStream_t s);
// Monitoring latent pass (state in the iterate type): also the latent parts of the residuals.
template <typename T, typename WT>
void latent_monitor_launch(const LatentArgs<T, WT>& a, int K, dim3 grid, unsigned threads, size_t smem,
                           cudaStream_t s);
// Dynamic shared-memory cap of the single-problem and batched latent kernels for patch size K.
template <typename T, typename WT>
cudaError_t latent_set_smem(int K, int bytes);
template <typename T, typename WT>
cudaError_t latent_batch_set_smem(int K, int bytes);

// ---- pixel updates and blur stencils (k_pixel.cuh, k_stencil.cuh) ----
// Pixel closed forms of one problem (register kernel for L_s <= 32, else the wide kernel).
template <typename T>
void pixel_launch(const PixelArgs<T>& a, unsigned blocks, unsigned threads, size_t smem, cudaStream_t s);
// Batched pixel closed forms (L_s <= 32).
template <typename T>
void pixel_batch_launch(const PixelArgs<T>* args, const Segment* seg, int nseg, int Ls, unsigned blocks,
                        size_t smem, cudaStream_t s);
// Blur stencil (MODE 0: B in; MODE 1: right-hand side).  sep_host: for a separable square blur,
// its factors in FP64, cu[bh] then cv[bh] (taps(u, v) = cu[u] cv[v]; separable kernel), else NULL;
// taps_host: the bh x bw taps in FP64 when bh == bw (the square kernel takes them as arguments),
// else NULL (generic kernel, taps read from a.taps).  smem: the 2D kernels' dynamic shared memory
// (the separable kernel sizes its own).
template <typename T, int MODE>
void stencil_launch(const StencilArgs<T>& a, int bh, const double* sep_host, const double* taps_host, dim3 grid,
                    size_t smem, cudaStream_t s);
// nbands: the bands of every problem (the separable kernel takes stencil_sep_bands per block; its
// segment table counts band groups, the other kernels' count bands).
template <typename T, int MODE>
void stencil_batch_launch(const StencilArgs<T>* args, const Segment* seg, int nseg, int bh, const double* sep_host,
                          const double* taps_host, unsigned blocks, size_t smem, cudaStream_t s, int nbands);
// Dynamic shared-memory cap of the stencil kernels for blur height bh and of the wide pixel kernel.
template <typename T>
cudaError_t pixel_stencil_set_smem(int bh, int bytes);
template <typename T>
cudaError_t stencil_batch_set_smem(int bh, int bytes);

// ---- register-resident DFT solve (k_wfft.cuh) ----
// One pass (0: rows forward, 1: columns with f, 2: rows inverse) over npair band pairs of one
// problem whose sides are wfft_length_ok; smem: the column pass's wfft_cols_smem<T>(H).
template <typename T>
void wfft_pass_launch(const FFTArgs<T>& a, int pass, int npair, size_t smem, cudaStream_t s);
// One pass over the segment table of a batch, each problem in the form its FFTArgs select
// (fT set: register-resident, ceil(H / 8) row blocks or ceil(W / 8) column blocks per pair;
// NULL: Stockham, the problem's rpb / CW shape); smem: the largest any block of the pass needs.
template <typename T>
void fft_batch_launch(const FFTArgs<T>* args, const Segment* seg, int nseg, int pass, unsigned blocks, size_t smem,
                      cudaStream_t s);
// Dynamic shared-memory cap of the register-form column kernels and the batched kernels.
template <typename T>
cudaError_t wfft_set_smem(int bytes);

// ---- reverse pass (k_grad.cuh) ----
template <typename T, typename WT>
void latent_bwd_tma_launch(const LatentBwdArgs<T, WT>& a, int K, dim3 grid, unsigned threads, size_t smem,
                           cudaStream_t s);
template <typename T, typename WT>
void latent_bwd_reg_launch(const T* X, const WT* omega, const T* Sin, T* Sb, const T* Rb, T* planes, double* part,
                           int H, int W, int Ls, int S, int Ty, T coef, int half, int K, dim3 grid, unsigned threads,
                           size_t smem, cudaStream_t s);
template <typename T, typename WT>
void omega_bwd_launch(const T* X, const WT* omega, const T* Sin, const T* Sb, const T* Rb, T* omega_bar, int H, int W,
                      int Ls, int S, T coef, T scale, int half, int K, dim3 grid, cudaStream_t s);
template <typename T>
void pixel_bwd_launch(const PixelBwdArgs<T>& a, unsigned blocks, cudaStream_t s);
template <typename T, typename WT>
cudaError_t latent_bwd_set_smem(int K, int bytes);

#define FUSE_LAUNCH_EXTERN_T_WT(T, WT)                                                                      \
    extern template void latent_tma_launch<T, WT>(const LatentArgs<T, WT>&, int, bool, dim3, unsigned, size_t,   \
                                                  cudaStream_t);                                               \
    extern template void latent_tma_batch_launch<T, WT>(const LatentArgs<T, WT>*, const Segment*, int, int, int, \
                                                        bool, unsigned, unsigned, size_t, cudaStream_t);       \
    extern template void latent_reg_launch<T, WT>(const T*, const WT*, const T*, T*, T*, int, int, int, int, int, \
                                                  T, int, int, dim3, unsigned, size_t, cudaStream_t);          \
    extern template void latent_monitor_launch<T, WT>(const LatentArgs<T, WT>&, int, dim3, unsigned, size_t,    \
                                                      cudaStream_t);                                           \
    extern template cudaError_t latent_set_smem<T, WT>(int, int);                                             \
    extern template cudaError_t latent_batch_set_smem<T, WT>(int, int);                                       \
    extern template void latent_bwd_tma_launch<T, WT>(const LatentBwdArgs<T, WT>&, int, dim3, unsigned, size_t, \
                                                      cudaStream_t);                                           \
    extern template void latent_bwd_reg_launch<T, WT>(const T*, const WT*, const T*, T*, const T*, T*, double*,  \
                                                      int, int, int, int, int, T, int, int, dim3, unsigned,     \
                                                      size_t, cudaStream_t);                                   \
    extern template void omega_bwd_launch<T, WT>(const T*, const WT*, const T*, const T*, const T*, T*, int, int,\
                                                 int, int, T, T, int, int, dim3, cudaStream_t);                \
    extern template cudaError_t latent_bwd_set_smem<T, WT>(int, int);

#define FUSE_LAUNCH_EXTERN_T(T)                                                                             \
    extern template void pixel_launch<T>(const PixelArgs<T>&, unsigned, unsigned, size_t, cudaStream_t);     \
    extern template void pixel_batch_launch<T>(const PixelArgs<T>*, const Segment*, int, int, unsigned, size_t, \
                                               cudaStream_t);                                                 \
    extern template void stencil_launch<T, 0>(const StencilArgs<T>&, int, const double*, const double*, dim3,  \
                                              size_t, cudaStream_t);                                          \
    extern template void stencil_launch<T, 1>(const StencilArgs<T>&, int, const double*, const double*, dim3,  \
                                              size_t, cudaStream_t);                                          \
    extern template void stencil_batch_launch<T, 0>(const StencilArgs<T>*, const Segment*, int, int,           \
                                                    const double*, const double*, unsigned, size_t,           \
                                                    cudaStream_t, int);                                            \
    extern template void stencil_batch_launch<T, 1>(const StencilArgs<T>*, const Segment*, int, int,           \
                                                    const double*, const double*, unsigned, size_t,           \
                                                    cudaStream_t, int);                                            \
    extern template cudaError_t pixel_stencil_set_smem<T>(int, int);                                          \
    extern template cudaError_t stencil_batch_set_smem<T>(int, int);                                          \
    extern template void pixel_bwd_launch<T>(const PixelBwdArgs<T>&, unsigned, cudaStream_t);                \
    extern template void wfft_pass_launch<T>(const FFTArgs<T>&, int, int, size_t, cudaStream_t);             \
    extern template void fft_batch_launch<T>(const FFTArgs<T>*, const Segment*, int, int, unsigned, size_t,   \
                                             cudaStream_t);                                                  \
    extern template cudaError_t wfft_set_smem<T>(int);

#ifndef FUSE_LAUNCH_DEFINITIONS
FUSE_LAUNCH_EXTERN_T_WT(float, float)
FUSE_LAUNCH_EXTERN_T_WT(float, __nv_bfloat16)
FUSE_LAUNCH_EXTERN_T_WT(double, double)
FUSE_LAUNCH_EXTERN_T(float)
FUSE_LAUNCH_EXTERN_T(double)
#endif

}  // namespace fuse
