// Launchers of the reverse-pass kernels (k_grad.cuh): the latent reverse (bulk-copy and
// register-staged), the weight adjoint and the pixel reverse, every instantiation compiled in
// this translation unit.
#define FUSE_LAUNCH_DEFINITIONS
#include "launch.cuh"

#include "dispatch.cuh"

namespace fuse {

template <typename T, typename WT>
void latent_bwd_tma_launch(const LatentBwdArgs<T, WT>& a, int K, dim3 grid, unsigned threads, size_t smem,
                           cudaStream_t s) {
    constexpr int VEC = 16 / sizeof(T);
    with_k(K, [&](auto k) { latent_bwd_tma_kernel<T, WT, decltype(k)::value, VEC><<<grid, threads, smem, s>>>(a); });
}

template <typename T, typename WT>
void latent_bwd_reg_launch(const T* X, const WT* omega, const T* Sin, T* Sb, const T* Rb, T* planes, double* part,
                           int H, int W, int Ls, int S, int Ty, T coef, int half, int K, dim3 grid, unsigned threads,
                           size_t smem, cudaStream_t s) {
    constexpr int VEC = 16 / sizeof(T);
    with_k(K, [&](auto k) {
        latent_bwd_kernel<T, WT, decltype(k)::value, VEC><<<grid, threads, smem, s>>>(X, omega, Sin, Sb, Rb, planes,
                                                                                       part, H, W, Ls, S, Ty, coef, half);
    });
}

template <typename T, typename WT>
void omega_bwd_launch(const T* X, const WT* omega, const T* Sin, const T* Sb, const T* Rb, T* omega_bar, int H, int W,
                      int Ls, int S, T coef, T scale, int half, int K, dim3 grid, cudaStream_t s) {
    with_k(K, [&](auto k) {
        omega_bwd_kernel<T, WT, decltype(k)::value><<<grid, 256, 0, s>>>(X, omega, Sin, Sb, Rb, omega_bar, H, W, Ls,
                                                                         S, coef, scale, half);
    });
}

template <typename T>
void pixel_bwd_launch(const PixelBwdArgs<T>& a, unsigned blocks, cudaStream_t s) {
    with_maxls(a.Ls, [&](auto m) {
        constexpr int M = decltype(m)::value;
        if constexpr (M > 0) pixel_bwd_kernel<T, M><<<blocks, 128, 0, s>>>(a);
    });
}

template <typename T, typename WT>
cudaError_t latent_bwd_set_smem(int K, int bytes) {
    constexpr int VEC = 16 / sizeof(T);
    const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    with_k(K, [&](auto k) {
        constexpr int KK = decltype(k)::value;
        e = cudaFuncSetAttribute(latent_bwd_kernel<T, WT, KK, VEC>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(latent_bwd_tma_kernel<T, WT, KK, VEC>, A, bytes);
    });
    return e;
}

#define FUSE_GRAD_INST_WT(T, WT)                                                                               \
    template void latent_bwd_tma_launch<T, WT>(const LatentBwdArgs<T, WT>&, int, dim3, unsigned, size_t,         \
                                               cudaStream_t);                                                  \
    template void latent_bwd_reg_launch<T, WT>(const T*, const WT*, const T*, T*, const T*, T*, double*, int, int, \
                                               int, int, int, T, int, int, dim3, unsigned, size_t, cudaStream_t); \
    template void omega_bwd_launch<T, WT>(const T*, const WT*, const T*, const T*, const T*, T*, int, int, int,   \
                                          int, T, T, int, int, dim3, cudaStream_t);                            \
    template cudaError_t latent_bwd_set_smem<T, WT>(int, int);

FUSE_GRAD_INST_WT(float, float)
FUSE_GRAD_INST_WT(float, __nv_bfloat16)
FUSE_GRAD_INST_WT(double, double)
template void pixel_bwd_launch<float>(const PixelBwdArgs<float>&, unsigned, cudaStream_t);
template void pixel_bwd_launch<double>(const PixelBwdArgs<double>&, unsigned, cudaStream_t);

}  // namespace fuse
