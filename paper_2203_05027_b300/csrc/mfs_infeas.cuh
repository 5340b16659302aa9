// mfs_infeas.cuh -- reductions for the infeasibility tests of mfs_solve, between two residual checks.
// Primal infeasible: d = lambda - lambda_prev and t = A^T d = s - s_prev (s = c + A^T lambda); by
// Farkas' lemma, A^T d in K* (= K) with b^T d < 0 certifies that Ax = b, x in K has no solution.
// Unbounded: e = x - x_prev with A e = 0, e in K and c^T e < 0 is a ray along which c^T x falls
// without end (then the dual has no solution).
#pragma once

#include <cuda_runtime.h>

namespace mfs {
namespace infeas {

// Per block, the sums (fixed order) for both tests, with t = s - s_prev, d = lambda - lambda_prev,
// e = x - x_prev and A e = r - r_prev (r = A x - b):
//   part[5 blk + 0] dist(t, K)^2 over orthant coordinates     part[5 blk + 1] ||d||^2
//   part[5 blk + 2] dist(e, K)^2 over orthant coordinates     part[5 blk + 3] ||e||^2
//   part[5 blk + 4] ||A e||^2
// Lorentz-cone coordinates are left to k_infeas_cones.
template <typename T>
__global__ void k_infeas(const double* __restrict__ s, const double* __restrict__ s_prev, const T* __restrict__ lam,
                         const double* __restrict__ lam_prev, const T* __restrict__ x, const double* __restrict__ x_prev,
                         const double* __restrict__ r, const double* __restrict__ r_prev,
                         const unsigned char* __restrict__ in_cone, int n, int m, double* __restrict__ part) {
    __shared__ double sh[5][256];
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const double e = double(x[j]) - x_prev[j];
        v[3] += e * e;
        if (!in_cone[j]) {
            const double t = s[j] - s_prev[j];
            v[0] += t < 0.0 ? t * t : 0.0;
            v[2] += e < 0.0 ? e * e : 0.0;
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double d = double(lam[i]) - lam_prev[i], ae = r[i] - r_prev[i];
        v[1] += d * d;
        v[4] += ae * ae;
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < 5; ++q) part[5 * blockIdx.x + q] = sh[q][0];
}

// dist(w, K_q)^2 for a Lorentz cone K_q and w = (w1, wbar), |wbar| = a, |wbar|^2 = aa
__device__ __forceinline__ double lorentz_dist2_of(double w1, double a, double aa) {
    if (a <= -w1) return aa + w1 * w1;  // w in the polar cone: its own norm
    if (a <= w1) return 0.0;
    return 0.5 * (a - w1) * (a - w1);
}

// Per Lorentz cone q: dist2[2q] = dist(t, K_q)^2, dist2[2q+1] = dist(e, K_q)^2 (one thread per cone).
template <typename T>
__global__ void k_infeas_cones(const double* __restrict__ s, const double* __restrict__ s_prev,
                               const T* __restrict__ x, const double* __restrict__ x_prev,
                               const int* __restrict__ soc_start, const int* __restrict__ soc_size, int nsoc,
                               double* __restrict__ dist2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsoc) return;
    const int st = soc_start[q], sz = soc_size[q];
    double tt = 0.0, ee = 0.0;
    for (int k = 1; k < sz; ++k) {
        const double t = s[st + k] - s_prev[st + k], e = double(x[st + k]) - x_prev[st + k];
        tt += t * t;
        ee += e * e;
    }
    dist2[2 * q] = lorentz_dist2_of(s[st] - s_prev[st], sqrt(tt), tt);
    dist2[2 * q + 1] = lorentz_dist2_of(double(x[st]) - x_prev[st], sqrt(ee), ee);
}

}  // namespace infeas
}  // namespace mfs
