// mfs_infeas.cuh -- reductions for the primal infeasibility test of mfs_solve: between two residual
// checks, d = lambda - lambda_prev and t = A^T d = s - s_prev with s = c + A^T lambda (FP64, from the
// residual kernels). By Farkas' lemma, A^T d in K* (= K) with b^T d < 0 certifies that Ax = b, x in K
// has no solution; these kernels give dist(t, K)^2 and ||d||^2 in a fixed order.
#pragma once

#include <cuda_runtime.h>

namespace mfs {
namespace infeas {

// Per block: sum over orthant coordinates of min(t_j, 0)^2 (dist(t, K)^2 there) and sum of
// d_i^2. Lorentz-cone coordinates are left to k_infeas_cones. part: [gridDim.x][2].
template <typename T>
__global__ void k_infeas(const double* __restrict__ s, const double* __restrict__ s_prev, const T* __restrict__ lam,
                         const double* __restrict__ lam_prev, const unsigned char* __restrict__ in_cone, int n, int m,
                         double* __restrict__ part) {
    __shared__ double sh[2][256];
    double a = 0.0, b = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        if (!in_cone[j]) {
            const double t = s[j] - s_prev[j];
            a += t < 0.0 ? t * t : 0.0;
        }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double d = double(lam[i]) - lam_prev[i];
        b += d * d;
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sh[0][0];
        part[2 * blockIdx.x + 1] = sh[1][0];
    }
}

// dist(t, K_q)^2 of each Lorentz cone q for t = s - s_prev (one thread per cone, into dist2[q]).
__global__ void k_infeas_cones(const double* __restrict__ s, const double* __restrict__ s_prev,
                               const int* __restrict__ soc_start, const int* __restrict__ soc_size, int nsoc,
                               double* __restrict__ dist2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsoc) return;
    const int st = soc_start[q], sz = soc_size[q];
    double tt = 0.0;
    for (int k = 1; k < sz; ++k) {
        const double t = s[st + k] - s_prev[st + k];
        tt += t * t;
    }
    const double t1 = s[st] - s_prev[st], a = sqrt(tt);
    double d2;
    if (a <= -t1)
        d2 = tt + t1 * t1;  // t in the polar cone: its own norm
    else if (a <= t1)
        d2 = 0.0;
    else
        d2 = 0.5 * (a - t1) * (a - t1);
    dist2[q] = d2;
}

}  // namespace infeas
}  // namespace mfs
