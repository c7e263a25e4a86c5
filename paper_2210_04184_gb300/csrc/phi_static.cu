// fuse_phi_static: the regulariser value phi(X) of eq. reg1 without any allocation.
//
// Who needs it: code that must not call cudaMalloc, for example a host application that
// gives the GPU a fixed memory budget and owns every allocation itself, or a loop with a
// latency bound that cannot afford the device synchronisation cudaMalloc may imply.  Such a
// caller cannot create a fuse_ctx (fuse_init allocates), so this entry point takes plain
// device pointers and keeps its only scratch - the per-block partial sums - in a file-scope
// device array of fixed size, resident on every GPU that loads the library until the process
// exits.
#include "fuse.h"

#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "k_objective.cuh"

namespace {

constexpr int kPhiStaticPartials = 1 << 18;      // 2 MiB of doubles
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_phi_scratch[kPhiStaticPartials];

// Per-device address of g_phi_scratch (host code only sees a host-side stand-in for the
// symbol, so the device address is looked up with that device current).  A successful lookup is
// kept; a failed one is not, so a later call tries again.
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

double* scratch_for(int dev) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_phi_scratch) != cudaSuccess) {
            cudaGetLastError();              // leave no pending error for the caller's next check
            return nullptr;
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    return g_scratch_ptr[dev];
}

// Sums the partial sums in a fixed order (deterministic) into out[0].
__global__ void __launch_bounds__(256) phi_static_reduce_kernel(const double* __restrict__ part, int count,
                                                               double* __restrict__ out) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < count; i += blockDim.x) v[0] += part[i];
    fuse::block_sum<1>(v, out);
}

}  // namespace

extern "C" fuse_status fuse_phi_static(const void* X_dev, const void* omega_dev, int H, int W, int L_s, int K,
                                       int S, fuse_dtype dtype, fuse_dtype wdtype, double* phi_dev,
                                       void* stream) {
    if (!X_dev || !omega_dev || !phi_dev) return FUSE_EINVAL;
    if (H < 1 || W < 1 || L_s < 1 || K < 0 || S < 1) return FUSE_EINVAL;
    if (2 * (K + S) + 1 > H || 2 * (K + S) + 1 > W) return FUSE_EINVAL;
    const bool f64 = dtype == FUSE_F64;
    if (dtype != FUSE_F32 && dtype != FUSE_F64) return FUSE_EINVAL;
    if (f64 && wdtype != FUSE_F64) return FUSE_EUNSUPPORTED;
    if (!f64 && wdtype != FUSE_F32 && wdtype != FUSE_BF16) return FUSE_EUNSUPPORTED;
    const size_t n = (size_t)H * W;
    const int nW = (2 * S + 1) * (2 * S + 1) - 1;
    const size_t nb = (n + 255) / 256;
    if (nb * (size_t)nW > (size_t)kPhiStaticPartials) return FUSE_EUNSUPPORTED;   // beyond the array

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FUSE_ECUDA;
    }
    double* part = scratch_for(dev);
    if (!part) return FUSE_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 grid((unsigned)nb, (unsigned)nW);
    // the regulariser kernel of fuse_objective, its partial sums written to the static array:
    // part[tau * nb + b] = sum over block b's pixels i of omega_tau(i) sum_{k, c} |D_{tau k} X(i, c)|;
    // every slot in [0, nb*nW) is written before the reduction reads it
    if (f64) {
        fuse::obj_phi_kernel<double, double><<<grid, 256, 0, s>>>(
            static_cast<const double*>(X_dev), static_cast<const double*>(omega_dev), H, W, L_s, K, S, part);
    } else if (wdtype == FUSE_BF16) {
        fuse::obj_phi_kernel<float, __nv_bfloat16><<<grid, 256, 0, s>>>(
            static_cast<const float*>(X_dev), static_cast<const __nv_bfloat16*>(omega_dev), H, W, L_s, K, S, part);
    } else {
        fuse::obj_phi_kernel<float, float><<<grid, 256, 0, s>>>(
            static_cast<const float*>(X_dev), static_cast<const float*>(omega_dev), H, W, L_s, K, S, part);
    }
    if (cudaGetLastError() != cudaSuccess) return FUSE_ECUDA;
    phi_static_reduce_kernel<<<1, 256, 0, s>>>(part, (int)(nb * nW), phi_dev);
    if (cudaGetLastError() != cudaSuccess) return FUSE_ECUDA;
    return FUSE_OK;
}
