// mfs_literal.cuh -- Algorithm 1 in its literal form, with the o-length splitting variables y and
// gamma, for a start from an arbitrary (x, y, z, gamma, delta, lambda). After two literal iterations
// the state satisfies gamma = -U^T lambda and y = V^T x + U^T F_U (b - A x) (the first from the
// y-step's optimality condition, the second once the y-step has seen a consistent gamma), and the
// solver continues with the reduced sweeps.
//
// The nonzeros are addressed in Algorithm 1's order k (columns in turn, rows ascending within a
// column): krow[k], kcol[k], kval[k]; perm lists the k of each row in ascending order (row i owns
// perm[rp[i] .. rp[i+1]-1]). One thread per column, nonzero or row; every sum runs in a fixed order.
#pragma once

#include <cuda_runtime.h>

namespace mfs {
namespace literal {

// k order from the chunked column layout: chunk c holds columns desc.x .. desc.y-1, whose nonzeros
// k = col_ptr[desc.x] + e sit at padded position desc.z + e.
template <typename T>
__global__ void k_kmap(const int* __restrict__ col_ptr, const int4* __restrict__ cdesc, int nchunks,
                       const int* __restrict__ cidx, const T* __restrict__ cval, int* __restrict__ krow,
                       int* __restrict__ kcol, T* __restrict__ kval) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    const int4 d = cdesc[c];
    const int k0 = col_ptr[d.x];
    for (int j = d.x; j < d.y; ++j)
        for (int k = col_ptr[j]; k < col_ptr[j + 1]; ++k) {
            const int p = d.z + (k - k0);
            krow[k] = cidx[p];
            kval[k] = cval[p];
            kcol[k] = j;
        }
}

// x-step: x_j = F_V,j ( sum_{k in column j} (y_k + gamma_k/mu) + z_j + delta_j/mu - c_j/mu )
template <typename T>
__global__ void k_x(const int* __restrict__ col_ptr, const T* __restrict__ y, const T* __restrict__ g,
                    const T* __restrict__ z, const T* __restrict__ del, const T* __restrict__ c, T mu,
                    T* __restrict__ x, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int k0 = col_ptr[j], k1 = col_ptr[j + 1];
    T s = T(0);
    for (int k = k0; k < k1; ++k) s += y[k] + g[k] / mu;
    const T fv = T(1) / (T(1) + T(k1 - k0));
    x[j] = fv * (s + z[j] + del[j] / mu - c[j] / mu);
}

// w = U^T (b - lambda/mu) + V^T x - gamma/mu, per nonzero
template <typename T>
__global__ void k_w(const int* __restrict__ krow, const int* __restrict__ kcol, const T* __restrict__ kval,
                    const T* __restrict__ b, const T* __restrict__ lam, const T* __restrict__ x,
                    const T* __restrict__ g, T mu, T* __restrict__ w, long long o) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < o; k += (long long)gridDim.x * blockDim.x) {
        const int i = krow[k];
        w[k] = kval[k] * (b[i] - lam[i] / mu) + x[kcol[k]] - g[k] / mu;
    }
}

// per row: out_i = F_U,i * sum_{k in row i} a_k u_k  (scale = 1) or  sum a_k u_k  (scale = 0)
template <typename T>
__global__ void k_rowdot(const int* __restrict__ rp, const int* __restrict__ perm, const T* __restrict__ kval,
                         const T* __restrict__ u, int fu_scale, T* __restrict__ out, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    T s = T(0), r = T(0);
    for (int q = rp[i]; q < rp[i + 1]; ++q) {
        const int k = perm[q];
        const T a = kval[k];
        s += a * u[k];
        r += a * a;
    }
    out[i] = fu_scale ? s / (T(1) + r) : s;
}

// y-step: y_k = w_k - a_k (F_U U w)_{i_k}
template <typename T>
__global__ void k_y(const int* __restrict__ krow, const T* __restrict__ kval, const T* __restrict__ w,
                    const T* __restrict__ fuw, T* __restrict__ y, long long o) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < o; k += (long long)gridDim.x * blockDim.x)
        y[k] = w[k] - kval[k] * fuw[krow[k]];
}

// argument of the z-step: x - delta/mu, in FP64 for the projection kernels
template <typename T>
__global__ void k_zarg(const T* __restrict__ x, const T* __restrict__ del, T mu, double* __restrict__ out, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = double(x[j] - del[j] / mu);
}

// dual updates: lambda += mu (U y - b) (uy = U y per row), gamma += mu (y - V^T x), delta += mu (z - x)
template <typename T>
__global__ void k_lam(const T* __restrict__ uy, const T* __restrict__ b, T mu, T* __restrict__ lam, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) lam[i] = lam[i] + mu * (uy[i] - b[i]);
}
template <typename T>
__global__ void k_gam(const int* __restrict__ kcol, const T* __restrict__ y, const T* __restrict__ x, T mu,
                      T* __restrict__ g, long long o) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < o; k += (long long)gridDim.x * blockDim.x)
        g[k] = g[k] + mu * (y[k] - x[kcol[k]]);
}
template <typename T>
__global__ void k_del(const T* __restrict__ z, const T* __restrict__ x, T mu, T* __restrict__ del, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) del[j] = del[j] + mu * (z[j] - x[j]);
}

}  // namespace literal
}  // namespace mfs
