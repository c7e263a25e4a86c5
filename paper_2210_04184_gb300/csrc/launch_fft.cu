// Launchers of the DFT solve's passes: the register-resident form (k_wfft.cuh), every (T, P)
// instantiation of its three passes, and the batched kernels of both forms are compiled in this
// translation unit.
#define FUSE_LAUNCH_DEFINITIONS
#include "launch.cuh"

namespace fuse {

template <typename T>
void wfft_pass_launch(const FFTArgs<T>& a, int pass, int npair, size_t smem, cudaStream_t s) {
    const int P = (pass == 1 ? a.H : a.W) / 32;
    const dim3 grid((unsigned)(pass == 1 ? (a.W + kWfftCols - 1) / kWfftCols : (a.H + 7) / 8), (unsigned)npair);
    switch (P) {
#define FUSE_WFFT_LAUNCH(PV)                                                                   \
        case PV:                                                                               \
            if (pass == 0) wfft_rows_fwd_kernel<T, PV><<<grid, 256, 0, s>>>(a);                \
            else if (pass == 1) wfft_cols_kernel<T, PV><<<grid, 256, smem, s>>>(a);            \
            else wfft_rows_inv_kernel<T, PV><<<grid, 256, 0, s>>>(a);                          \
            break;
        FUSE_WFFT_CASES(FUSE_WFFT_LAUNCH)
#undef FUSE_WFFT_LAUNCH
        default: break;
    }
}

template <typename T>
void fft_batch_launch(const FFTArgs<T>* args, const Segment* seg, int nseg, int pass, unsigned blocks, size_t smem,
                      cudaStream_t s) {
    if (pass == 0) fft_batch_kernel<T, 0><<<blocks, 256, smem, s>>>(args, seg, nseg);
    else if (pass == 1) fft_batch_kernel<T, 1><<<blocks, 256, smem, s>>>(args, seg, nseg);
    else fft_batch_kernel<T, 2><<<blocks, 256, smem, s>>>(args, seg, nseg);
}

template <typename T>
cudaError_t wfft_set_smem(int bytes) {
    const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(fft_batch_kernel<T, 0>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fft_batch_kernel<T, 1>, A, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fft_batch_kernel<T, 2>, A, bytes);
#define FUSE_WFFT_ATTR(PV) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(wfft_cols_kernel<T, PV>, A, bytes);
    FUSE_WFFT_CASES(FUSE_WFFT_ATTR)
#undef FUSE_WFFT_ATTR
    return e;
}

template void wfft_pass_launch<float>(const FFTArgs<float>&, int, int, size_t, cudaStream_t);
template void wfft_pass_launch<double>(const FFTArgs<double>&, int, int, size_t, cudaStream_t);
template void fft_batch_launch<float>(const FFTArgs<float>*, const Segment*, int, int, unsigned, size_t, cudaStream_t);
template void fft_batch_launch<double>(const FFTArgs<double>*, const Segment*, int, int, unsigned, size_t,
                                       cudaStream_t);
template cudaError_t wfft_set_smem<float>(int);
template cudaError_t wfft_set_smem<double>(int);

}  // namespace fuse
