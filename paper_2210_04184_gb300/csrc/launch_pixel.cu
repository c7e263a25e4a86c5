// Launchers of the pixel closed forms (k_pixel.cuh) and the blur stencils (k_stencil.cuh):
// every (T, MAXLS) and (T, MODE, blur size) instantiation is compiled in this translation unit.
#define FUSE_LAUNCH_DEFINITIONS
#include "launch.cuh"

#include "dispatch.cuh"

namespace fuse {

template <typename T>
void pixel_launch(const PixelArgs<T>& a, unsigned blocks, unsigned threads, size_t smem, cudaStream_t s) {
    with_maxls(a.Ls, [&](auto m) {
        constexpr int M = decltype(m)::value;
        if constexpr (M == 0) pixel_kernel_wide<T><<<blocks, threads, smem, s>>>(a);
        else pixel_kernel<T, M><<<blocks, threads, smem, s>>>(a);
    });
}

template <typename T>
void pixel_batch_launch(const PixelArgs<T>* args, const Segment* seg, int nseg, int Ls, unsigned blocks, size_t smem,
                        cudaStream_t s) {
    with_maxls(Ls, [&](auto m) {
        constexpr int M = decltype(m)::value;
        if constexpr (M != 0) pixel_batch_kernel<T, M><<<blocks, 128, smem, s>>>(args, seg, nseg);
    });
}

template <typename T, int B>
SepTaps<T, B> sep_taps(const double* sep_host) {
    SepTaps<T, B> tp;
    for (int i = 0; i < B; ++i) {
        tp.cu[i] = (T)sep_host[i];
        tp.cv[i] = (T)sep_host[B + i];
    }
    return tp;
}

template <typename T, int MODE>
void stencil_launch(const StencilArgs<T>& a, int bh, const double* sep_host, const double* taps_host, dim3 grid,
                    size_t smem, cudaStream_t s) {
    if (sep_host) {
        // grid.z counts bands; the separable kernel takes stencil_sep_bands of them per block
        constexpr int NB = stencil_sep_bands<T, MODE>();
        const int nbands = (int)grid.z;
        const dim3 g(grid.x, grid.y, (unsigned)((nbands + NB - 1) / NB));
        with_bh(bh, [&](auto b) {
            constexpr int B = decltype(b)::value;
            stencil_sep_kernel<T, MODE, B><<<g, dim3(ST_TX, ST_BY), stencil_sep_smem<T, B, NB>(), s>>>(
                a, sep_taps<T, B>(sep_host), nbands);
        });
        return;
    }
    if (taps_host) {
        with_bh(bh, [&](auto b) {
            constexpr int B = decltype(b)::value;
            SquareTaps<T, B> tp;
            for (int i = 0; i < B * B; ++i) tp.t[i] = (T)taps_host[i];
            stencil_sq_kernel<T, MODE, B><<<grid, dim3(ST_TX, ST_BY), smem, s>>>(a, tp);
        });
        return;
    }
    with_bh(bh, [&](auto b) {
        stencil_kernel<T, MODE, decltype(b)::value><<<grid, dim3(ST_TX, ST_BY), smem, s>>>(a);
    });
}

template <typename T, int MODE>
void stencil_batch_launch(const StencilArgs<T>* args, const Segment* seg, int nseg, int bh, const double* sep_host,
                          const double* taps_host, unsigned blocks, size_t smem, cudaStream_t s, int nbands) {
    if (sep_host) {
        constexpr int NB = stencil_sep_bands<T, MODE>();
        with_bh(bh, [&](auto b) {
            constexpr int B = decltype(b)::value;
            stencil_sep_batch_kernel<T, MODE, B><<<blocks, dim3(ST_TX, ST_BY), stencil_sep_smem<T, B, NB>(), s>>>(
                args, seg, nseg, sep_taps<T, B>(sep_host), nbands);
        });
        return;
    }
    if (taps_host) {
        with_bh(bh, [&](auto b) {
            constexpr int B = decltype(b)::value;
            SquareTaps<T, B> tp;
            for (int i = 0; i < B * B; ++i) tp.t[i] = (T)taps_host[i];
            stencil_sq_batch_kernel<T, MODE, B><<<blocks, dim3(ST_TX, ST_BY), smem, s>>>(args, seg, nseg, tp);
        });
        return;
    }
    with_bh(bh, [&](auto b) {
        stencil_batch_kernel<T, MODE, decltype(b)::value><<<blocks, dim3(ST_TX, ST_BY), smem, s>>>(args, seg, nseg);
    });
}

template <typename T>
cudaError_t pixel_stencil_set_smem(int bh, int bytes) {
    const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(pixel_kernel_wide<T>, A, bytes);
    with_bh(bh, [&](auto b) {
        constexpr int B = decltype(b)::value;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<T, 0, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_kernel<T, 1, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_sq_kernel<T, 0, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_sq_kernel<T, 1, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_sep_kernel<T, 0, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_sep_kernel<T, 1, B>, A, bytes);
    });
    return e;
}

template <typename T>
cudaError_t stencil_batch_set_smem(int bh, int bytes) {
    const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    with_bh(bh, [&](auto b) {
        constexpr int B = decltype(b)::value;
        e = cudaFuncSetAttribute(stencil_batch_kernel<T, 0, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_batch_kernel<T, 1, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_sq_batch_kernel<T, 0, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_sq_batch_kernel<T, 1, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_sep_batch_kernel<T, 0, B>, A, bytes);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(stencil_sep_batch_kernel<T, 1, B>, A, bytes);
    });
    return e;
}

#define FUSE_PIXEL_INST(T)                                                                                     \
    template void pixel_launch<T>(const PixelArgs<T>&, unsigned, unsigned, size_t, cudaStream_t);               \
    template void pixel_batch_launch<T>(const PixelArgs<T>*, const Segment*, int, int, unsigned, size_t,        \
                                        cudaStream_t);                                                          \
    template void stencil_launch<T, 0>(const StencilArgs<T>&, int, const double*, const double*, dim3, size_t,   \
                                       cudaStream_t);                                                           \
    template void stencil_launch<T, 1>(const StencilArgs<T>&, int, const double*, const double*, dim3, size_t,   \
                                       cudaStream_t);                                                           \
    template void stencil_batch_launch<T, 0>(const StencilArgs<T>*, const Segment*, int, int, const double*,     \
                                             const double*, unsigned, size_t, cudaStream_t, int);               \
    template void stencil_batch_launch<T, 1>(const StencilArgs<T>*, const Segment*, int, int, const double*,     \
                                             const double*, unsigned, size_t, cudaStream_t, int);               \
    template cudaError_t pixel_stencil_set_smem<T>(int, int);                                                   \
    template cudaError_t stencil_batch_set_smem<T>(int, int);

FUSE_PIXEL_INST(float)
FUSE_PIXEL_INST(double)

}  // namespace fuse
