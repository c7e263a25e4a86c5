// Launchers of the forward latent pass (k_latent.cuh): every (T, WT, K) instantiation of the
// bulk-copy, batched and register-staged kernels is compiled in this translation unit.
#define FUSE_LAUNCH_DEFINITIONS
#include "launch.cuh"

#include "dispatch.cuh"

namespace fuse {

template <typename T, typename WT>
void latent_tma_launch(const LatentArgs<T, WT>& a, int K, bool int16_state, dim3 grid, unsigned threads,
                       size_t smem, cudaStream_t s) {
    constexpr int TVEC = 32 / sizeof(T);
    with_k(K, [&](auto k) {
        constexpr int KK = decltype(k)::value;
        if constexpr (sizeof(T) == 4) {
            if (int16_state) {
                latent_tma_kernel<T, WT, KK, TVEC, int16_t><<<grid, threads, smem, s>>>(a);
                return;
            }
        }
        latent_tma_kernel<T, WT, KK, TVEC><<<grid, threads, smem, s>>>(a);
    });
}

template <typename T, typename WT>
void latent_tma_batch_launch(const LatentArgs<T, WT>* args, const Segment* seg, int nseg, int zero_in, int K,
                             bool int16_state, unsigned blocks, unsigned threads, size_t smem, cudaStream_t s) {
    constexpr int TVEC = 32 / sizeof(T);
    with_k(K, [&](auto k) {
        constexpr int KK = decltype(k)::value;
        if constexpr (sizeof(T) == 4) {
            if (int16_state) {
                latent_tma_batch_kernel<T, WT, KK, TVEC, int16_t><<<blocks, threads, smem, s>>>(args, seg, nseg, zero_in);
                return;
            }
        }
        latent_tma_batch_kernel<T, WT, KK, TVEC><<<blocks, threads, smem, s>>>(args, seg, nseg, zero_in);
    });
}

template <typename T, typename WT>
void latent_monitor_launch(const LatentArgs<T, WT>& a, int K, dim3 grid, unsigned threads, size_t smem,
                           cudaStream_t s) {
    constexpr int TVEC = 32 / sizeof(T);
    with_k(K, [&](auto k) { latent_tma_monitor_kernel<T, WT, decltype(k)::value, TVEC><<<grid, threads, smem, s>>>(a); });
}

template <typename T, typename WT>
void latent_reg_launch(const T* X, const WT* omega, const T* Sig, T* Sout, T* planes, int H, int W, int Ls, int S,
                       int Ty, T coef, int half, int K, dim3 grid, unsigned threads, size_t smem, cudaStream_t s) {
    constexpr int VEC = 16 / sizeof(T);
    with_k(K, [&](auto k) {
        latent_kernel<T, WT, decltype(k)::value, VEC><<<grid, threads, smem, s>>>(X, omega, Sig, Sout, planes, H, W,
                                                                                   Ls, S, Ty, coef, half);
    });
}

template <typename T, typename WT>
cudaError_t latent_set_smem(int K, int bytes) {
    constexpr int VEC = 16 / sizeof(T), TVEC = 32 / sizeof(T);
    const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    with_k(K, [&](auto k) {
        constexpr int KK = decltype(k)::value;
        e = cudaFuncSetAttribute(latent_kernel<T, WT, KK, VEC>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(latent_tma_kernel<T, WT, KK, TVEC>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(latent_tma_monitor_kernel<T, WT, KK, TVEC>, A, bytes);
        if constexpr (sizeof(T) == 4) {
            if (e == cudaSuccess) e = cudaFuncSetAttribute(latent_tma_kernel<T, WT, KK, TVEC, int16_t>, A, bytes);
        }
    });
    return e;
}

template <typename T, typename WT>
cudaError_t latent_batch_set_smem(int K, int bytes) {
    constexpr int TVEC = 32 / sizeof(T);
    const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    with_k(K, [&](auto k) {
        constexpr int KK = decltype(k)::value;
        e = cudaFuncSetAttribute(latent_tma_batch_kernel<T, WT, KK, TVEC>, A, bytes);
        if constexpr (sizeof(T) == 4) {
            if (e == cudaSuccess) e = cudaFuncSetAttribute(latent_tma_batch_kernel<T, WT, KK, TVEC, int16_t>, A, bytes);
        }
    });
    return e;
}

#define FUSE_LATENT_INST(T, WT)                                                                               \
    template void latent_tma_launch<T, WT>(const LatentArgs<T, WT>&, int, bool, dim3, unsigned, size_t,          \
                                           cudaStream_t);                                                      \
    template void latent_tma_batch_launch<T, WT>(const LatentArgs<T, WT>*, const Segment*, int, int, int, bool,  \
                                                 unsigned, unsigned, size_t, cudaStream_t);                    \
    template void latent_monitor_launch<T, WT>(const LatentArgs<T, WT>&, int, dim3, unsigned, size_t,            \
                                               cudaStream_t);                                                  \
    template void latent_reg_launch<T, WT>(const T*, const WT*, const T*, T*, T*, int, int, int, int, int, T,    \
                                           int, int, dim3, unsigned, size_t, cudaStream_t);                    \
    template cudaError_t latent_set_smem<T, WT>(int, int);                                                      \
    template cudaError_t latent_batch_set_smem<T, WT>(int, int);

FUSE_LATENT_INST(float, float)
FUSE_LATENT_INST(float, __nv_bfloat16)
FUSE_LATENT_INST(double, double)

}  // namespace fuse
