// ADMM residual norms of one iteration (Sec. IV, scaled form of the splitting of eq. fusionoptim:
// constraint A X = z with A = (B; I; D_{tau k}), z = (P1, P2, Q), scaled duals Lambda1, Lambda2,
// Sigma):
//   primal  ||A X' - z'|| = sqrt(||B X' - P1'||^2 + ||X' - P2'||^2 + sum ||D X' - Q'||^2)
//   dual    rho ||A^T (z' - z)|| = rho ||B^T dP1 + dP2 + sum D^T dQ||
// The dual updates (eqs. dualvar1_main..dualvar3_main) give B X' - P1' = Lambda1 - Lambda1',
// X' - P2' = Lambda2 - Lambda2' and D X' - Q' = Sigma - Sigma', so the primal residual is the
// change of the scaled duals.  The kernels keep U = P + Lambda, so dP = (U' - Lambda') - (U - Lambda).
// sum D^T dQ comes from the latent pass's adjoint planes: with the planes R of sum D^T (Q + Sigma)
// (entering the iteration) and M of sum D^T (Q' + Sigma) (the monitoring latent pass),
// sum D^T dQ = M - R.
#pragma once
#include "common.cuh"
#include "k_objective.cuh"

namespace fuse {

// Per block: sum of (Lambda1' - Lambda1)^2 + (Lambda2' - Lambda2)^2; dP1 and dP2 written over the
// saved U1 and U2 (U1o <- dP1, U2o <- dP2).  Grid-stride over the count = L_s n elements.
template <typename T>
__global__ void __launch_bounds__(256)
monitor_pixel_kernel(const T* __restrict__ L1, const T* __restrict__ U1, const T* __restrict__ L2,
                     const T* __restrict__ U2, const T* __restrict__ L1o, T* __restrict__ U1o,
                     const T* __restrict__ L2o, T* __restrict__ U2o, size_t count, double* __restrict__ part) {
    double v[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const T l1 = L1[i], l2 = L2[i], a1 = L1o[i], a2 = L2o[i];
        const double d1 = (double)(l1 - a1), d2 = (double)(l2 - a2);
        v[0] += d1 * d1 + d2 * d2;
        U1o[i] = (U1[i] - l1) - (U1o[i] - a1);
        U2o[i] = (U2[i] - l2) - (U2o[i] - a2);
    }
    block_sum<1>(v, part + blockIdx.x);
}

// a <- a - b (grid-stride)
template <typename T>
__global__ void __launch_bounds__(256) sub_kernel(T* __restrict__ a, const T* __restrict__ b, size_t count) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        a[i] -= b[i];
}

// Per block: sum of a^2 in FP64 (grid-stride).
template <typename T>
__global__ void __launch_bounds__(256) sumsq_kernel(const T* __restrict__ a, size_t count, double* __restrict__ part) {
    double v[1] = {0.0};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const double x = (double)a[i];
        v[0] += x * x;
    }
    block_sum<1>(v, part + blockIdx.x);
}

}  // namespace fuse
