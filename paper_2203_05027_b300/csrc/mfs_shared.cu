// mfs_shared.cu -- many problems that share one constraint matrix A and differ in b and c (the
// mfs_shared_* calls of include/mfs.h): Algorithm 1 on B instances at once.
//
// The instances' vectors are interleaved, x[j * Bp + s] for instance s (Bp = B rounded up to 32),
// so one warp serves one column (or row) for 32 instances: the warp reads the column's nonzeros
// once (broadcast) and each gather of the other side's vector is one coalesced 128-byte load of 32
// instances' values. Each iteration is the reduced form of the single-instance solver:
//   column sweep  x = F_V (d x + A^T v + z + (delta - c)/mu), z = proj_K(x - delta/mu),
//                 delta += mu (z - x);
//   row sweep     rho = F_U (b - A x), lambda -= mu rho, v = rho - lambda/mu.
// Residuals are reduced per instance in FP64 (per-nonzero products as exact FP32 pairs).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/mfs.h"
#include "mfs_trace.h"
#include "mfs_alloc.h"
#include "mfs_device.cuh"
#include "mfs_measures.h"

namespace {

using mfs::DF;
using mfs::FULL;

constexpr int SNT = 256;           // threads per CTA
constexpr int SW = SNT / 32;       // warps per CTA
constexpr int NSTAT = 23;

template <typename T>
struct SArgs {
    int m, n, Bp;
    const int* col_ptr;
    const int* cidx;
    const T* cval;
    const int* row_ptr;
    const int* ridx;
    const T* rval;
    const T* fu;            // F_U = 1 / (1 + sum_k a_ik^2) per row
    const unsigned char* in_soc;  // per column: 1 if in a Lorentz cone
    int nsoc;
    const int* soc_start;
    const int* soc_size;
    const T* b;  // [m][Bp]
    const T* c;  // [n][Bp]
    T* x;
    T* z;
    T* del;
    T* lam;
    T* v;
    T mu;
};

template <typename T>
__device__ __forceinline__ T lorentz_coord(T w, int t, T w1, T alpha) {
    if (alpha <= -w1) return T(0);
    if (alpha <= w1) return w;
    return (t == 0) ? w / T(2) + alpha / T(2) : w / T(2) + w1 * w / (T(2) * alpha);
}

__device__ __forceinline__ double lorentz_dist2(double w1, double alpha, double wnorm2) {
    if (alpha <= -w1) return wnorm2;
    if (alpha <= w1) return 0.0;
    const double g = alpha - w1;
    return 0.5 * g * g;
}

// V consecutive instances per lane: vector loads and stores of the interleaved state.
template <typename T, int V>
struct alignas(sizeof(T) * V) Pack {
    T e[V];
};
template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ld_pack(const T* p) {
    return *reinterpret_cast<const Pack<T, V>*>(p);
}
template <typename T, int V>
__device__ __forceinline__ void st_pack(T* p, const Pack<T, V>& v) {
    *reinterpret_cast<Pack<T, V>*>(p) = v;
}
// read-only gather of V instances (the gathered vector is not written by the same launch)
template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ldg_pack(const T* p) {
    Pack<T, V> r;
    if constexpr (V == 4 && sizeof(T) == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        r.e[0] = q.x, r.e[1] = q.y, r.e[2] = q.z, r.e[3] = q.w;
    } else if constexpr (V == 2 && sizeof(T) == 4) {
        const float2 q = __ldg(reinterpret_cast<const float2*>(p));
        r.e[0] = q.x, r.e[1] = q.y;
    } else if constexpr (V == 2 && sizeof(T) == 8) {
        const double2 q = __ldg(reinterpret_cast<const double2*>(p));
        r.e[0] = q.x, r.e[1] = q.y;
    } else {
        static_assert(V == 1, "unsupported pack");
        r.e[0] = __ldg(p);
    }
    return r;
}

// acc[u] = sum over the nonzeros k of a line (column or row) of val[k] * g[idx[k] * Bp + s0 + u]:
// the warp loads 32 indices and values at a time with one coalesced load each, broadcasts them by
// shuffles and keeps GIF gathers in flight; the sum runs in the nonzeros' order.
#ifndef MFS_SHARED_GIF
#define MFS_SHARED_GIF 4
#endif
constexpr int GIF = MFS_SHARED_GIF;
template <typename T, int V>
__device__ __forceinline__ void line_dot(const int* __restrict__ idx, const T* __restrict__ val, int k0, int k1,
                                         const T* __restrict__ g, int Bp, int s0, int lane, T (&acc)[V]) {
#pragma unroll
    for (int u = 0; u < V; ++u) acc[u] = T(0);
    for (int base = k0; base < k1; base += 32) {
        const int cnt = min(32, k1 - base);
        int mi = 0;
        T mv = T(0);
        if (lane < cnt) {
            mi = __ldg(idx + base + lane);
            mv = __ldg(val + base + lane);
        }
        int t = 0;
        for (; t + GIF <= cnt; t += GIF) {
            Pack<T, V> q[GIF];
            T w[GIF];
#pragma unroll
            for (int r = 0; r < GIF; ++r) {
                const int i = __shfl_sync(FULL, mi, t + r);
                w[r] = __shfl_sync(FULL, mv, t + r);
                q[r] = ldg_pack<T, V>(g + (size_t)i * Bp + s0);
            }
#pragma unroll
            for (int r = 0; r < GIF; ++r)
#pragma unroll
                for (int u = 0; u < V; ++u) acc[u] += w[r] * q[r].e[u];
        }
        for (; t < cnt; ++t) {
            const int i = __shfl_sync(FULL, mi, t);
            const T w = __shfl_sync(FULL, mv, t);
            const Pack<T, V> q = ldg_pack<T, V>(g + (size_t)i * Bp + s0);
#pragma unroll
            for (int u = 0; u < V; ++u) acc[u] += w * q.e[u];
        }
    }
}

// one warp per (column, group of 32 V instances); lane takes instances s0 .. s0+V-1
template <typename T, int V>
__global__ void __launch_bounds__(SNT) k_s_col(const SArgs<T> a) {
    const long long w = (long long)blockIdx.x * SW + (threadIdx.x >> 5);
    const int groups = a.Bp / (32 * V), lane = threadIdx.x & 31;
    if (w >= (long long)a.n * groups) return;
    // group-major: all columns of one group of instances before the next, so that the gathered
    // slice of v (m x 32V values) stays in L2 while it is used
    const int j = (int)(w % a.n);
    const int s0 = (int)(w / a.n) * 32 * V + lane * V;
    const int k0 = a.col_ptr[j], k1 = a.col_ptr[j + 1];
    T acc[V];
    line_dot<T, V>(a.cidx, a.cval, k0, k1, a.v, a.Bp, s0, lane, acc);
    const size_t p = (size_t)j * a.Bp + s0;
    const T d = T(k1 - k0), mu = a.mu;
    const Pack<T, V> xo = ld_pack<T, V>(a.x + p), zo = ld_pack<T, V>(a.z + p), dl = ld_pack<T, V>(a.del + p),
                     cc = ld_pack<T, V>(a.c + p);
    Pack<T, V> xn, zn, dn;
#pragma unroll
    for (int u = 0; u < V; ++u) xn.e[u] = (d * xo.e[u] + acc[u] + zo.e[u] + (dl.e[u] - cc.e[u]) / mu) / (T(1) + d);
    st_pack<T, V>(a.x + p, xn);
    if (!a.in_soc[j]) {
#pragma unroll
        for (int u = 0; u < V; ++u) {
            const T wv = xn.e[u] - dl.e[u] / mu;
            zn.e[u] = wv > T(0) ? wv : T(0);
            dn.e[u] = dl.e[u] + mu * (zn.e[u] - xn.e[u]);
        }
        st_pack<T, V>(a.z + p, zn);
        st_pack<T, V>(a.del + p, dn);
    }
}

// z-step and delta-update of Lorentz cones: one warp per (cone, slice); x holds the new x
template <typename T>
__global__ void __launch_bounds__(SNT) k_s_cone(const SArgs<T> a) {
    const long long w = (long long)blockIdx.x * SW + (threadIdx.x >> 5);
    const int slices = a.Bp >> 5;
    if (w >= (long long)a.nsoc * slices) return;
    const int q = (int)(w / slices);
    const int s = (int)(w % slices) * 32 + (threadIdx.x & 31);
    const int st = a.soc_start[q], sz = a.soc_size[q];
    const T mu = a.mu;
    T ss = T(0);
    for (int t = 1; t < sz; ++t) {
        const size_t p = (size_t)(st + t) * a.Bp + s;
        const T wv = a.x[p] - a.del[p] / mu;
        ss += wv * wv;
    }
    const size_t p0 = (size_t)st * a.Bp + s;
    const T alpha = sqrt(ss), w1 = a.x[p0] - a.del[p0] / mu;
    for (int t = 0; t < sz; ++t) {
        const size_t p = (size_t)(st + t) * a.Bp + s;
        const T xt = a.x[p], dt = a.del[p];
        const T zt = lorentz_coord(xt - dt / mu, t, w1, alpha);
        a.z[p] = zt;
        a.del[p] = dt + mu * (zt - xt);
    }
}

// one warp per (row, group of 32 V instances). MODE 0: iteration; MODE 1: v from x and the
// current lambda.
template <typename T, int MODE, int V>
__global__ void __launch_bounds__(SNT) k_s_row(const SArgs<T> a) {
    const long long w = (long long)blockIdx.x * SW + (threadIdx.x >> 5);
    const int groups = a.Bp / (32 * V), lane = threadIdx.x & 31;
    if (w >= (long long)a.m * groups) return;
    const int i = (int)(w % a.m);  // group-major, as in k_s_col (the gathered slice of x stays in L2)
    const int s0 = (int)(w / a.m) * 32 * V + lane * V;
    T acc[V];
    line_dot<T, V>(a.ridx, a.rval, a.row_ptr[i], a.row_ptr[i + 1], a.x, a.Bp, s0, lane, acc);
    const size_t p = (size_t)i * a.Bp + s0;
    const T mu = a.mu, fu = a.fu[i];
    const Pack<T, V> bb = ld_pack<T, V>(a.b + p), lo = ld_pack<T, V>(a.lam + p);
    Pack<T, V> ln, vn;
#pragma unroll
    for (int u = 0; u < V; ++u) {
        const T rho = (bb.e[u] - acc[u]) * fu;
        ln.e[u] = MODE == 0 ? lo.e[u] - mu * rho : lo.e[u];
        vn.e[u] = rho - ln.e[u] / mu;
    }
    if (MODE == 0) st_pack<T, V>(a.lam + p, ln);
    st_pack<T, V>(a.v + p, vn);
}

template <typename T>
struct AccT {
    using type = DF;
};
template <>
struct AccT<double> {
    using type = double;
};
__device__ __forceinline__ DF acc_mul(float x, float y) { return mfs::df_prod(x, y); }
__device__ __forceinline__ double acc_mul(double x, double y) { return x * y; }

enum { RES2, RESMAX, AXMAX, B2, BMAX, BLAM, S2, SMAX, ATLMAX, C2, CMAX, CX, X2, SDIST2, XDIST2, XMAX, SDMAX, XDMAX, NFLD };
__host__ __device__ constexpr bool is_max(int f) {
    return f == RESMAX || f == AXMAX || f == BMAX || f == SMAX || f == ATLMAX || f == CMAX || f == XMAX || f == SDMAX ||
           f == XDMAX;
}

// Per-instance residual fields. grid (G, Bp/32); warp w of block (g, q) takes rows (columns,
// cones) g*SW + w, + G*SW, ...; lane = instance. Partials part[f][g][s]; s_out (nullable) gets
// c + A^T lambda per (j, s).
template <typename T>
__global__ void __launch_bounds__(SNT) k_s_resid(const SArgs<T> a, double* part, T* s_out) {
    using A = typename AccT<T>::type;
    __shared__ double sh[SW][NFLD][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.y * 32 + lane;
    const int G = gridDim.x;
    double f[NFLD];
#pragma unroll
    for (int k = 0; k < NFLD; ++k) f[k] = 0.0;
    for (int i = blockIdx.x * SW + warp; i < a.m; i += G * SW) {
        A acc = A(0);
        for (int k = a.row_ptr[i]; k < a.row_ptr[i + 1]; ++k) acc = acc + acc_mul(a.rval[k], a.x[(size_t)a.ridx[k] * a.Bp + s]);
        const size_t p = (size_t)i * a.Bp + s;
        const double ax = mfs::to_double(acc), bi = double(a.b[p]), res = ax - bi;
        f[RES2] += res * res;
        f[RESMAX] = fmax(f[RESMAX], fabs(res));
        f[AXMAX] = fmax(f[AXMAX], fabs(ax));
        f[B2] += bi * bi;
        f[BMAX] = fmax(f[BMAX], fabs(bi));
        f[BLAM] += bi * double(a.lam[p]);
    }
    auto column = [&](int j) {
        A acc = A(0);
        for (int k = a.col_ptr[j]; k < a.col_ptr[j + 1]; ++k) acc = acc + acc_mul(a.cval[k], a.lam[(size_t)a.cidx[k] * a.Bp + s]);
        const size_t p = (size_t)j * a.Bp + s;
        const double atl = mfs::to_double(acc), cj = double(a.c[p]), xj = double(a.x[p]);
        const double sv = cj + atl;
        f[S2] += sv * sv;
        f[SMAX] = fmax(f[SMAX], fabs(sv));
        f[ATLMAX] = fmax(f[ATLMAX], fabs(atl));
        f[C2] += cj * cj;
        f[CMAX] = fmax(f[CMAX], fabs(cj));
        f[CX] += cj * xj;
        f[X2] += xj * xj;
        f[XMAX] = fmax(f[XMAX], fabs(xj));
        if (s_out) s_out[p] = T(sv);
        return sv;
    };
    for (int j = blockIdx.x * SW + warp; j < a.n; j += G * SW) {
        const double sv = column(j);
        if (!a.in_soc[j]) {
            const double xj = double(a.x[(size_t)j * a.Bp + s]);
            const double sn = sv < 0.0 ? sv : 0.0, xn = xj < 0.0 ? xj : 0.0;
            f[SDIST2] += sn * sn;
            f[XDIST2] += xn * xn;
            f[SDMAX] = fmax(f[SDMAX], -sn);
            f[XDMAX] = fmax(f[XDMAX], -xn);
        }
    }
    for (int q = blockIdx.x * SW + warp; q < a.nsoc; q += G * SW) {
        // the cone's columns were counted above; here only its distances, recomputing s
        const int st = a.soc_start[q], sz = a.soc_size[q];
        double s1 = 0, ss = 0, x1 = 0, xx = 0;
        for (int t = 0; t < sz; ++t) {
            const int j = st + t;
            A acc = A(0);
            for (int k = a.col_ptr[j]; k < a.col_ptr[j + 1]; ++k)
                acc = acc + acc_mul(a.cval[k], a.lam[(size_t)a.cidx[k] * a.Bp + s]);
            const size_t p = (size_t)j * a.Bp + s;
            const double sv = double(a.c[p]) + mfs::to_double(acc), xj = double(a.x[p]);
            if (t == 0) {
                s1 = sv;
                x1 = xj;
            } else {
                ss += sv * sv;
                xx += xj * xj;
            }
        }
        f[SDIST2] += lorentz_dist2(s1, sqrt(ss), ss + s1 * s1);
        f[XDIST2] += lorentz_dist2(x1, sqrt(xx), xx + x1 * x1);
        f[SDMAX] = fmax(f[SDMAX], mfs::lorentz_distinf(s1, sqrt(ss)));
        f[XDMAX] = fmax(f[XDMAX], mfs::lorentz_distinf(x1, sqrt(xx)));
    }
#pragma unroll
    for (int k = 0; k < NFLD; ++k) sh[warp][k][lane] = f[k];
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < NFLD; ++k) {
            double acc = 0.0;
            for (int w = 0; w < SW; ++w) acc = is_max(k) ? fmax(acc, sh[w][k][lane]) : acc + sh[w][k][lane];
            part[((size_t)k * G + blockIdx.x) * a.Bp + s] = acc;
        }
    }
}

__global__ void k_s_finalize(const double* part, int G, int Bp, int B, double* status) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    double f[NFLD];
    for (int k = 0; k < NFLD; ++k) {
        double acc = 0.0;
        for (int g = 0; g < G; ++g) {
            const double v = part[((size_t)k * G + g) * Bp + s];
            acc = is_max(k) ? ((v > acc || v != v) ? v : acc) : acc + v;
        }
        f[k] = acc;
    }
    const double nres = sqrt(f[RES2]), nb = sqrt(f[B2]), nxd = sqrt(f[XDIST2]), nx = sqrt(f[X2]);
    const double nsd = sqrt(f[SDIST2]), nc = sqrt(f[C2]), cx = f[CX], bl = f[BLAM];
    double* st = status + (size_t)s * NSTAT;
    st[0] = nres / (1.0 + nb);
    st[1] = nsd / (1.0 + nc);
    st[2] = nxd / (1.0 + nx);
    st[3] = fabs(cx + bl) / (1.0 + fabs(cx) + fabs(bl));
    double kkt = st[0];
    for (int q = 1; q < 4; ++q) kkt = (st[q] > kkt || st[q] != st[q]) ? st[q] : kkt;
    st[4] = kkt;
    st[5] = cx;
    st[6] = -bl;
    st[7] = nres;
    st[8] = nb;
    st[9] = nxd;
    st[10] = nx;
    st[11] = nsd;
    st[12] = nc;
    st[13] = sqrt(f[S2]);
    st[14] = f[RESMAX];
    st[15] = f[AXMAX];
    st[16] = f[BMAX];
    st[17] = f[SMAX];
    st[18] = f[ATLMAX];
    st[19] = f[CMAX];
    st[20] = f[XMAX];
    st[21] = f[XDMAX];
    st[22] = f[SDMAX];
}

// [count][len] instance-major (FP32 or FP64 source) -> [len][Bp] interleaved T, and back.
template <typename S, typename D>
__global__ void k_s_interleave(const S* __restrict__ src, D* __restrict__ dst, int count, int len, int Bp) {
    __shared__ D tile[32][33];
    const int l0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int s = s0 + k, l = l0 + threadIdx.x;
        tile[k][threadIdx.x] = (s < count && l < len) ? D(src[(size_t)s * len + l]) : D(0);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int l = l0 + k, s = s0 + threadIdx.x;
        if (l < len && s < Bp) dst[(size_t)l * Bp + s] = tile[threadIdx.x][k];
    }
}
template <typename S, typename D>
__global__ void k_s_deinterleave(const S* __restrict__ src, D* __restrict__ dst, int count, int len, int Bp) {
    __shared__ S tile[32][33];
    const int l0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int l = l0 + k, s = s0 + threadIdx.x;
        tile[k][threadIdx.x] = (l < len && s < Bp) ? src[(size_t)l * Bp + s] : S(0);
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int s = s0 + k, l = l0 + threadIdx.x;
        if (s < count && l < len) dst[(size_t)s * len + l] = D(tile[threadIdx.x][k]);
    }
}

// out = proj_K(in) per instance (interleaved): orthant coordinates elementwise, cones per warp/slice
template <typename T>
__global__ void k_s_proj_orthant(const T* __restrict__ in, T* __restrict__ out, const unsigned char* in_soc, int n, int Bp) {
    const long long total = (long long)n * Bp;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / Bp);
        if (!in_soc[j]) out[t] = in[t] > T(0) ? in[t] : T(0);
    }
}
template <typename T>
__global__ void k_s_proj_cones(const T* __restrict__ in, T* __restrict__ out, const int* soc_start, const int* soc_size,
                               int nsoc, int Bp) {
    const long long w = (long long)blockIdx.x * SW + (threadIdx.x >> 5);
    const int slices = Bp >> 5;
    if (w >= (long long)nsoc * slices) return;
    const int q = (int)(w / slices);
    const int s = (int)(w % slices) * 32 + (threadIdx.x & 31);
    const int st = soc_start[q], sz = soc_size[q];
    T ss = T(0);
    for (int t = 1; t < sz; ++t) {
        const T u = in[(size_t)(st + t) * Bp + s];
        ss += u * u;
    }
    const T alpha = sqrt(ss), w1 = in[(size_t)st * Bp + s];
    for (int t = 0; t < sz; ++t) {
        const size_t p = (size_t)(st + t) * Bp + s;
        out[p] = lorentz_coord(in[p], t, w1, alpha);
    }
}

// out[l] = src[l * Bp + t] (one instance of an interleaved array), as double
template <typename S>
__global__ void k_s_extract(const S* __restrict__ src, double* __restrict__ out, int len, int Bp, int t) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < len; l += gridDim.x * blockDim.x)
        out[l] = double(src[(size_t)l * Bp + t]);
}

// Slots of the interleaved layout, for members entering and leaving one at a time:
// dst[l][slots[q]] = src[q][l] (enter), dst[q][l] = src[l][slots[q]] (leave), arr[l][slots[q]] = 0.
template <typename S, typename D>
__global__ void k_s_scatter_slots(const S* __restrict__ src, D* __restrict__ dst, const int* __restrict__ slots,
                                  int count, int len, int Bp) {
    const long long total = (long long)count * len;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / len), l = (int)(t % len);
        dst[(size_t)l * Bp + slots[q]] = D(src[t]);
    }
}
template <typename S, typename D>
__global__ void k_s_gather_slots(const S* __restrict__ src, D* __restrict__ dst, const int* __restrict__ slots,
                                 int count, int len, int Bp) {
    const long long total = (long long)count * len;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / len), l = (int)(t % len);
        dst[t] = D(src[(size_t)l * Bp + slots[q]]);
    }
}
template <typename T>
__global__ void k_s_zero_slots(T* __restrict__ arr, const int* __restrict__ slots, int count, int len, int Bp) {
    const long long total = (long long)count * len;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
        arr[(size_t)(t % len) * Bp + slots[t / len]] = T(0);
}

// Warm start of single slots: projections of those slots only (orthant coordinates per (j, slot),
// Lorentz cones per (cone, slot)), and v = F_U (b - A x) - lambda/mu of those slots.
template <typename T>
__global__ void k_s_proj_slots_orthant(const T* __restrict__ in, T* __restrict__ out, const unsigned char* in_soc, int n,
                                       int Bp, const int* __restrict__ slots, int count) {
    const long long total = (long long)n * count;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / count);
        if (in_soc[j]) continue;
        const size_t p = (size_t)j * Bp + slots[t % count];
        out[p] = in[p] > T(0) ? in[p] : T(0);
    }
}
template <typename T>
__global__ void k_s_proj_slots_cones(const T* __restrict__ in, T* __restrict__ out, const int* soc_start,
                                     const int* soc_size, int nsoc, int Bp, const int* __restrict__ slots, int count) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nsoc * count) return;
    const int q = (int)(t / count), s = slots[t % count];
    const int st = soc_start[q], sz = soc_size[q];
    T ss = T(0);
    for (int k = 1; k < sz; ++k) {
        const T u = in[(size_t)(st + k) * Bp + s];
        ss += u * u;
    }
    const T alpha = sqrt(ss), w1 = in[(size_t)st * Bp + s];
    for (int k = 0; k < sz; ++k) {
        const size_t p = (size_t)(st + k) * Bp + s;
        out[p] = lorentz_coord(in[p], k, w1, alpha);
    }
}
template <typename T>
__global__ void k_s_row_slots(const SArgs<T> a, const int* __restrict__ slots, int count) {
    const long long total = (long long)a.m * count;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / count), s = slots[t % count];
        T acc = T(0);
        for (int k = a.row_ptr[i]; k < a.row_ptr[i + 1]; ++k) acc += a.rval[k] * a.x[(size_t)a.ridx[k] * a.Bp + s];
        const size_t p = (size_t)i * a.Bp + s;
        const T rho = (a.b[p] - acc) * a.fu[i];
        a.v[p] = rho - a.lam[p] / a.mu;
    }
}

template <typename T>
struct SStore {
    T *cval = nullptr, *rval = nullptr, *fu = nullptr, *b = nullptr, *c = nullptr;
    T *x = nullptr, *z = nullptr, *del = nullptr, *lam = nullptr, *v = nullptr, *sbuf = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
};

}  // namespace

struct mfs_shared {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mfs_settings set{};
    int m = 0, n = 0, o = 0, B = 0, Bp = 0, nsoc = 0, G = 1;
    int64_t iter = 0;
    int *col_ptr = nullptr, *cidx = nullptr, *row_ptr = nullptr, *ridx = nullptr, *soc_start = nullptr,
        *soc_size = nullptr;
    unsigned char* in_soc = nullptr;
    double *part = nullptr, *status = nullptr, *h_status = nullptr;
    int* slot_buf = nullptr;  // device copy of a slot list (B entries at most)
    SStore<float> f32;
    SStore<double> f64;
    std::vector<void*> allocs;
    std::string last_error;
};

namespace {

thread_local std::string g_shared_error;

mfs_status sfail(mfs_shared* s, mfs_status st, const std::string& msg) {
    if (s)
        s->last_error = msg;
    else
        g_shared_error = msg;
    return st;
}

#define SCUDA(s, call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return sfail((s), e_ == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA,         \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)
#define STRY(x)                         \
    do {                                \
        mfs_status st_ = (x);           \
        if (st_ != MFS_OK) return st_;  \
    } while (0)

template <typename T>
mfs_status salloc(mfs_shared* s, T** p, size_t count, const void* host = nullptr) {
    void* q = nullptr;
    SCUDA(s, mfs::device_malloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
    s->allocs.push_back(q);
    *p = static_cast<T*>(q);
    if (host && count)
        SCUDA(s, cudaMemcpyAsync(q, host, count * sizeof(T), cudaMemcpyHostToDevice, s->stream));
    else
        SCUDA(s, cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), s->stream));
    return MFS_OK;
}

template <typename T>
SArgs<T> sargs(mfs_shared* s, SStore<T>& st) {
    SArgs<T> a;
    a.m = s->m;
    a.n = s->n;
    a.Bp = s->Bp;
    a.col_ptr = s->col_ptr;
    a.cidx = s->cidx;
    a.cval = st.cval;
    a.row_ptr = s->row_ptr;
    a.ridx = s->ridx;
    a.rval = st.rval;
    a.fu = st.fu;
    a.in_soc = s->in_soc;
    a.nsoc = s->nsoc;
    a.soc_start = s->soc_start;
    a.soc_size = s->soc_size;
    a.b = st.b;
    a.c = st.c;
    a.x = st.x;
    a.z = st.z;
    a.del = st.del;
    a.lam = st.lam;
    a.v = st.v;
    a.mu = T(s->set.mu);
    return a;
}

inline int wgrid(long long warps) {
    return (int)((warps + SW - 1) / SW);
}

// instances per lane: the widest pack (16 bytes at most) that divides the interleave width
template <typename T>
int pack_of(int Bp) {
    if (sizeof(T) == 4 && Bp % 128 == 0) return 4;
    if (Bp % 64 == 0) return 2;
    return 1;
}

template <typename T, int V>
void s_iteration_v(mfs_shared* s, const SArgs<T>& a, cudaStream_t st) {
    const long long g = s->Bp / (32 * V);
    if (s->n) k_s_col<T, V><<<wgrid((long long)s->n * g), SNT, 0, st>>>(a);
    if (s->nsoc) k_s_cone<T><<<wgrid((long long)s->nsoc * (s->Bp / 32)), SNT, 0, st>>>(a);
    if (s->m) k_s_row<T, 0, V><<<wgrid((long long)s->m * g), SNT, 0, st>>>(a);
}

template <typename T>
void s_iteration(mfs_shared* s, const SArgs<T>& a, cudaStream_t st) {
    switch (pack_of<T>(s->Bp)) {
        case 4:
            if constexpr (sizeof(T) == 4) s_iteration_v<T, 4>(s, a, st);
            break;
        case 2: s_iteration_v<T, 2>(s, a, st); break;
        default: s_iteration_v<T, 1>(s, a, st);
    }
}

template <typename T>
void s_row_v(mfs_shared* s, const SArgs<T>& a) {
    if (!s->m) return;
    switch (pack_of<T>(s->Bp)) {
        case 4:
            if constexpr (sizeof(T) == 4)
                k_s_row<T, 1, 4><<<wgrid((long long)s->m * (s->Bp / 128)), SNT, 0, s->stream>>>(a);
            break;
        case 2: k_s_row<T, 1, 2><<<wgrid((long long)s->m * (s->Bp / 64)), SNT, 0, s->stream>>>(a); break;
        default: k_s_row<T, 1, 1><<<wgrid((long long)s->m * (s->Bp / 32)), SNT, 0, s->stream>>>(a);
    }
}

template <typename T>
mfs_status s_run(mfs_shared* s, SStore<T>& st, int64_t k) {
    SArgs<T> a = sargs(s, st);
    const int K = std::max(1, (int)s->set.check_every);
    if (k >= K) {
        if (!st.graph || st.graph_iters != K) {
            if (st.graph) cudaGraphExecDestroy(st.graph);
            st.graph = nullptr;
            cudaStream_t cap;
            SCUDA(s, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                for (int i = 0; i < K; ++i) s_iteration(s, a, cap);
                e = cudaStreamEndCapture(cap, &g);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&st.graph, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) {
                st.graph = nullptr;
                return sfail(s, MFS_ERR_CUDA, std::string("shared graph: ") + cudaGetErrorString(e));
            }
            st.graph_iters = K;
        }
        while (k >= K) {
            SCUDA(s, cudaGraphLaunch(st.graph, s->stream));
            k -= K;
            s->iter += K;
        }
    }
    for (int64_t i = 0; i < k; ++i) s_iteration(s, a, s->stream);
    s->iter += k;
    SCUDA(s, cudaGetLastError());
    return MFS_OK;
}

template <typename T>
mfs_status s_residuals(mfs_shared* s, SStore<T>& st, T* s_out) {
    SArgs<T> a = sargs(s, st);
    k_s_resid<T><<<dim3(s->G, s->Bp / 32), SNT, 0, s->stream>>>(a, s->part, s_out);
    k_s_finalize<<<(s->B + 127) / 128, 128, 0, s->stream>>>(s->part, s->G, s->Bp, s->B, s->status);
    SCUDA(s, cudaGetLastError());
    return MFS_OK;
}

template <typename T>
mfs_status s_alloc_store(mfs_shared* s, SStore<T>& st, const std::vector<double>& cv, const std::vector<double>& rv,
                         const std::vector<double>& fu) {
    std::vector<T> tmp(cv.begin(), cv.end());
    STRY(salloc(s, &st.cval, tmp.size(), tmp.data()));
    tmp.assign(rv.begin(), rv.end());
    STRY(salloc(s, &st.rval, tmp.size(), tmp.data()));
    tmp.assign(fu.begin(), fu.end());
    STRY(salloc(s, &st.fu, tmp.size(), tmp.data()));
    const size_t nb = (size_t)s->n * s->Bp, mb = (size_t)s->m * s->Bp;
    STRY(salloc(s, &st.b, mb));
    STRY(salloc(s, &st.c, nb));
    STRY(salloc(s, &st.x, nb));
    STRY(salloc(s, &st.z, nb));
    STRY(salloc(s, &st.del, nb));
    STRY(salloc(s, &st.sbuf, nb));
    STRY(salloc(s, &st.lam, mb));
    STRY(salloc(s, &st.v, mb));
    return MFS_OK;
}

template <typename S, typename D>
void interleave(const S* src, D* dst, int count, int len, int Bp, cudaStream_t st) {
    dim3 grid((len + 31) / 32, (Bp + 31) / 32), block(32, 8);
    k_s_interleave<S, D><<<grid, block, 0, st>>>(src, dst, count, len, Bp);
}
template <typename S, typename D>
void deinterleave(const S* src, D* dst, int count, int len, int Bp, cudaStream_t st) {
    dim3 grid((len + 31) / 32, (Bp + 31) / 32), block(32, 8);
    k_s_deinterleave<S, D><<<grid, block, 0, st>>>(src, dst, count, len, Bp);
}

template <typename T>
void s_destroy_graph(SStore<T>& st) {
    if (st.graph) cudaGraphExecDestroy(st.graph);
    st.graph = nullptr;
}

// Warm start from instance-major device arrays x [B][n], lambda [B][m] (FP32 or FP64 source S).
template <typename T, typename S>
mfs_status s_warm(mfs_shared* s, SStore<T>& st, const S* x, const S* lam) {
    const int sl = s->Bp / 32;
    interleave(x, st.x, s->B, s->n, s->Bp, s->stream);
    interleave(lam, st.lam, s->B, s->m, s->Bp, s->stream);
    const long long nb = (long long)s->n * s->Bp;
    const int g1 = (int)std::min<long long>((nb + 255) / 256, 148 * 16);
    // z = proj_K(x)
    if (s->n) k_s_proj_orthant<T><<<g1, 256, 0, s->stream>>>(st.x, st.z, s->in_soc, s->n, s->Bp);
    if (s->nsoc) k_s_proj_cones<T><<<wgrid((long long)s->nsoc * sl), SNT, 0, s->stream>>>(st.x, st.z, s->soc_start, s->soc_size, s->nsoc, s->Bp);
    // delta = proj_K(c + A^T lambda)
    STRY(s_residuals(s, st, st.sbuf));
    if (s->n) k_s_proj_orthant<T><<<g1, 256, 0, s->stream>>>(st.sbuf, st.del, s->in_soc, s->n, s->Bp);
    if (s->nsoc) k_s_proj_cones<T><<<wgrid((long long)s->nsoc * sl), SNT, 0, s->stream>>>(st.sbuf, st.del, s->soc_start, s->soc_size, s->nsoc, s->Bp);
    // v = F_U (b - A x) - lambda/mu
    SArgs<T> a = sargs(s, st);
    s_row_v(s, a);
    SCUDA(s, cudaGetLastError());
    SCUDA(s, cudaStreamSynchronize(s->stream));
    s->iter = 0;
    return MFS_OK;
}

}  // namespace

// Copies a host slot list to the device after checking it (distinct slots in [0, B)).
static mfs_status put_slots(mfs_shared* s, int64_t count, const int32_t* slots) {
    if (count < 0 || count > s->B || (count && !slots)) return sfail(s, MFS_ERR_INVALID, "slots: 0 <= count <= B");
    std::vector<char> seen(s->B, 0);
    for (int64_t q = 0; q < count; ++q) {
        if (slots[q] < 0 || slots[q] >= s->B || seen[slots[q]])
            return sfail(s, MFS_ERR_INVALID, "slots must be distinct and in [0, count of the handle)");
        seen[slots[q]] = 1;
    }
    if (count)
        SCUDA(s, cudaMemcpyAsync(s->slot_buf, slots, count * sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
    return MFS_OK;
}

static int grid_for(long long total) {
    return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 148LL * 16));
}

template <typename T>
static mfs_status load_slots_t(mfs_shared* s, SStore<T>& st, int count, const float* b, const float* c) {
    const int* sl = s->slot_buf;
    const long long tm = (long long)count * s->m, tn = (long long)count * s->n;
    if (tm) k_s_scatter_slots<float, T><<<grid_for(tm), 256, 0, s->stream>>>(b, st.b, sl, count, s->m, s->Bp);
    if (tn) k_s_scatter_slots<float, T><<<grid_for(tn), 256, 0, s->stream>>>(c, st.c, sl, count, s->n, s->Bp);
    T* nvec[3] = {st.x, st.z, st.del};
    T* mvec[2] = {st.lam, st.v};
    if (tn) {
        for (int q = 0; q < 3; ++q) k_s_zero_slots<T><<<grid_for(tn), 256, 0, s->stream>>>(nvec[q], sl, count, s->n, s->Bp);
    }
    if (tm) {
        for (int q = 0; q < 2; ++q) k_s_zero_slots<T><<<grid_for(tm), 256, 0, s->stream>>>(mvec[q], sl, count, s->m, s->Bp);
    }
    SCUDA(s, cudaGetLastError());
    return MFS_OK;
}

template <typename T>
static mfs_status warm_slots_t(mfs_shared* s, SStore<T>& st, int count, const float* x, const float* lam) {
    const int* sl = s->slot_buf;
    const long long tm = (long long)count * s->m, tn = (long long)count * s->n;
    if (tn) k_s_scatter_slots<float, T><<<grid_for(tn), 256, 0, s->stream>>>(x, st.x, sl, count, s->n, s->Bp);
    if (tm) k_s_scatter_slots<float, T><<<grid_for(tm), 256, 0, s->stream>>>(lam, st.lam, sl, count, s->m, s->Bp);
    // z = proj_K(x)
    if (tn) k_s_proj_slots_orthant<T><<<grid_for(tn), 256, 0, s->stream>>>(st.x, st.z, s->in_soc, s->n, s->Bp, sl, count);
    if (s->nsoc)
        k_s_proj_slots_cones<T><<<(int)((s->nsoc * (long long)count + 255) / 256), 256, 0, s->stream>>>(
            st.x, st.z, s->soc_start, s->soc_size, s->nsoc, s->Bp, sl, count);
    // delta = proj_K(c + A^T lambda): s = c + A^T lambda for all slots, projected for these
    STRY(s_residuals(s, st, st.sbuf));
    if (tn) k_s_proj_slots_orthant<T><<<grid_for(tn), 256, 0, s->stream>>>(st.sbuf, st.del, s->in_soc, s->n, s->Bp, sl, count);
    if (s->nsoc)
        k_s_proj_slots_cones<T><<<(int)((s->nsoc * (long long)count + 255) / 256), 256, 0, s->stream>>>(
            st.sbuf, st.del, s->soc_start, s->soc_size, s->nsoc, s->Bp, sl, count);
    // v = F_U (b - A x) - lambda/mu of these slots
    if (tm) k_s_row_slots<T><<<grid_for(tm), 256, 0, s->stream>>>(sargs(s, st), sl, count);
    SCUDA(s, cudaGetLastError());
    return MFS_OK;
}

extern "C" {

mfs_status mfs_shared_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val,
                             int64_t ncones, const mfs_cone* cones, int64_t count, const mfs_settings* settings,
                             void* cuda_stream, mfs_shared** out) {
    MFS_TRACE("mfs_shared_create");
    g_shared_error.clear();
    if (!out) return sfail(nullptr, MFS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (m < 0 || n < 0 || nnz < 0 || ncones < 0 || count < 1 || m >= INT32_MAX || n >= INT32_MAX || nnz >= INT32_MAX ||
        count > (1 << 20))
        return sfail(nullptr, MFS_ERR_INVALID, "bad sizes");
    if ((nnz && (!row || !col || !val)) || (ncones && !cones)) return sfail(nullptr, MFS_ERR_INVALID, "NULL array");
    mfs_settings set;
    mfs_default_settings(&set);
    if (settings) set = *settings;
    if (!(set.mu > 0.0) || !std::isfinite(set.mu) || set.check_every < 1 ||
        (set.precision != MFS_FP64 && set.precision != MFS_FP32_MIXED))
        return sfail(nullptr, MFS_ERR_INVALID, "invalid settings");
    std::vector<unsigned char> insoc(n, 0);
    std::vector<int> sst, ssz;
    int64_t covered = 0;
    for (int64_t q = 0; q < ncones; ++q) {
        if (cones[q].size < 1 || (cones[q].kind != MFS_CONE_NONNEG && cones[q].kind != MFS_CONE_SOC))
            return sfail(nullptr, MFS_ERR_INVALID, "bad cone");
        if (cones[q].kind == MFS_CONE_SOC) {
            sst.push_back((int)covered);
            ssz.push_back((int)cones[q].size);
            for (int64_t t = 0; t < cones[q].size; ++t) insoc[covered + t] = 1;
        }
        covered += cones[q].size;
    }
    if (covered != n) return sfail(nullptr, MFS_ERR_INVALID, "cone sizes do not sum to n");
    // column order (rows ascending), duplicates summed, zeros dropped; row order; F_U
    std::vector<int64_t> idx(nnz);
    std::iota(idx.begin(), idx.end(), 0);
    for (int64_t k = 0; k < nnz; ++k)
        if (row[k] < 0 || row[k] >= m || col[k] < 0 || col[k] >= n || !std::isfinite(val[k]))
            return sfail(nullptr, MFS_ERR_INVALID, "bad entry " + std::to_string(k));
    std::sort(idx.begin(), idx.end(),
              [&](int64_t p, int64_t q) { return col[p] != col[q] ? col[p] < col[q] : row[p] < row[q]; });
    std::vector<int> cp(n + 1, 0), ci, rp(m + 1, 0), ri;
    std::vector<double> cv, rv, fu(m, 0.0);
    std::vector<int> lc;
    for (int64_t k = 0; k < nnz;) {
        const int64_t r = row[idx[k]], q = col[idx[k]];
        double a = 0.0;
        while (k < nnz && row[idx[k]] == r && col[idx[k]] == q) a += val[idx[k++]];
        if (a != 0.0) {
            ci.push_back((int)r);
            cv.push_back(a);
            lc.push_back((int)q);
            cp[q + 1]++;
        }
    }
    for (int64_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
    const int o = (int)cv.size();
    for (int k = 0; k < o; ++k) {
        rp[ci[k] + 1]++;
        fu[ci[k]] += cv[k] * cv[k];
    }
    for (int64_t i = 0; i < m; ++i) rp[i + 1] += rp[i];
    for (int64_t i = 0; i < m; ++i) fu[i] = 1.0 / (1.0 + fu[i]);
    ri.resize(o);
    rv.resize(o);
    {
        std::vector<int> fill(rp.begin(), rp.begin() + m);
        for (int k = 0; k < o; ++k) {
            const int d = fill[ci[k]]++;
            ri[d] = lc[k];
            rv[d] = cv[k];
        }
    }
    mfs_shared* s = new (std::nothrow) mfs_shared();
    if (!s) return sfail(nullptr, MFS_ERR_OOM, "host allocation failed");
    auto bail = [&](mfs_status st) {
        g_shared_error = s->last_error;
        mfs_shared_destroy(s);
        return st;
    };
    s->set = set;
    s->m = (int)m;
    s->n = (int)n;
    s->o = o;
    s->B = (int)count;
    s->Bp = (int)((count + 31) / 32 * 32);
    s->nsoc = (int)sst.size();
    cudaError_t e = cudaGetDevice(&s->device);
    int sms = 148;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) {
        if (cuda_stream)
            s->stream = static_cast<cudaStream_t>(cuda_stream);
        else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = true;
        }
    }
    if (e != cudaSuccess) {
        s->last_error = std::string("CUDA set-up: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
    s->G = std::max(1, std::min((std::max(s->m, s->n) + SW - 1) / SW, 2 * sms / std::max(1, s->Bp / 32) + 1));
#define SCHK(x)                             \
    do {                                    \
        mfs_status q_ = (x);                \
        if (q_ != MFS_OK) return bail(q_);  \
    } while (0)
    SCHK(salloc(s, &s->col_ptr, cp.size(), cp.data()));
    SCHK(salloc(s, &s->cidx, ci.size(), ci.data()));
    SCHK(salloc(s, &s->row_ptr, rp.size(), rp.data()));
    SCHK(salloc(s, &s->ridx, ri.size(), ri.data()));
    SCHK(salloc(s, &s->in_soc, insoc.size(), insoc.data()));
    SCHK(salloc(s, &s->soc_start, sst.size(), sst.data()));
    SCHK(salloc(s, &s->soc_size, ssz.size(), ssz.data()));
    SCHK(salloc(s, &s->part, (size_t)NFLD * s->G * s->Bp));
    SCHK(salloc(s, &s->status, (size_t)NSTAT * s->B));
    SCHK(salloc(s, &s->slot_buf, (size_t)s->B));
    if (set.precision == MFS_FP64)
        SCHK(s_alloc_store(s, s->f64, cv, rv, fu));
    else
        SCHK(s_alloc_store(s, s->f32, cv, rv, fu));
    e = cudaMallocHost(&s->h_status, (size_t)NSTAT * s->B * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        s->last_error = std::string("set-up: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
#undef SCHK
    *out = s;
    return MFS_OK;
}

void mfs_shared_destroy(mfs_shared* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    s_destroy_graph(s->f32);
    s_destroy_graph(s->f64);
    for (void* p : s->allocs) cudaFree(p);
    if (s->h_status) cudaFreeHost(s->h_status);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char* mfs_shared_last_error(const mfs_shared* s) {
    return s ? s->last_error.c_str() : g_shared_error.c_str();
}

static mfs_status shared_set_data(mfs_shared* s, const void* b, const void* c, bool dbl, bool host) {
    if (!s || (s->m && !b) || (s->n && !c)) return MFS_ERR_INVALID;
    SCUDA(s, cudaSetDevice(s->device));
    const void *db = b, *dc = c;
    void* tmp = nullptr;
    const size_t es = dbl ? sizeof(double) : sizeof(float);
    if (host) {
        SCUDA(s, cudaMallocAsync(&tmp, std::max<size_t>(1, (size_t)s->B * (s->m + s->n) * es), s->stream));
        SCUDA(s, cudaMemcpyAsync(tmp, b, (size_t)s->B * s->m * es, cudaMemcpyHostToDevice, s->stream));
        char* tc = static_cast<char*>(tmp) + (size_t)s->B * s->m * es;
        SCUDA(s, cudaMemcpyAsync(tc, c, (size_t)s->B * s->n * es, cudaMemcpyHostToDevice, s->stream));
        db = tmp;
        dc = tc;
    }
    if (s->set.precision == MFS_FP64) {
        if (dbl) {
            interleave(static_cast<const double*>(db), s->f64.b, s->B, s->m, s->Bp, s->stream);
            interleave(static_cast<const double*>(dc), s->f64.c, s->B, s->n, s->Bp, s->stream);
        } else {
            interleave(static_cast<const float*>(db), s->f64.b, s->B, s->m, s->Bp, s->stream);
            interleave(static_cast<const float*>(dc), s->f64.c, s->B, s->n, s->Bp, s->stream);
        }
    } else {
        if (dbl) {
            interleave(static_cast<const double*>(db), s->f32.b, s->B, s->m, s->Bp, s->stream);
            interleave(static_cast<const double*>(dc), s->f32.c, s->B, s->n, s->Bp, s->stream);
        } else {
            interleave(static_cast<const float*>(db), s->f32.b, s->B, s->m, s->Bp, s->stream);
            interleave(static_cast<const float*>(dc), s->f32.c, s->B, s->n, s->Bp, s->stream);
        }
    }
    if (tmp) cudaFreeAsync(tmp, s->stream);
    SCUDA(s, cudaGetLastError());
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return mfs_shared_reset(s);
}

/* b [count][m], c [count][n] host doubles */
mfs_status mfs_shared_set_data(mfs_shared* s, const double* b, const double* c) {
    return shared_set_data(s, b, c, true, true);
}
/* same from device FP32 arrays */
mfs_status mfs_shared_set_data_device(mfs_shared* s, const float* b, const float* c) {
    return shared_set_data(s, b, c, false, false);
}

mfs_status mfs_shared_reset(mfs_shared* s) {
    if (!s) return MFS_ERR_INVALID;
    SCUDA(s, cudaSetDevice(s->device));
    const size_t nb = (size_t)s->n * s->Bp, mb = (size_t)s->m * s->Bp;
    if (s->set.precision == MFS_FP64) {
        for (double* p : {s->f64.x, s->f64.z, s->f64.del}) SCUDA(s, cudaMemsetAsync(p, 0, nb * sizeof(double), s->stream));
        for (double* p : {s->f64.lam, s->f64.v}) SCUDA(s, cudaMemsetAsync(p, 0, mb * sizeof(double), s->stream));
    } else {
        for (float* p : {s->f32.x, s->f32.z, s->f32.del}) SCUDA(s, cudaMemsetAsync(p, 0, nb * sizeof(float), s->stream));
        for (float* p : {s->f32.lam, s->f32.v}) SCUDA(s, cudaMemsetAsync(p, 0, mb * sizeof(float), s->stream));
    }
    SCUDA(s, cudaStreamSynchronize(s->stream));
    s->iter = 0;
    return MFS_OK;
}

/* warm start from device FP32 arrays x [count][n], lambda [count][m]; z = proj_K(x),
   delta = proj_K(c + A^T lambda) */
mfs_status mfs_shared_warm_start_device(mfs_shared* s, const float* x, const float* lambda) {
    if (!s || (s->n && !x) || (s->m && !lambda)) return MFS_ERR_INVALID;
    SCUDA(s, cudaSetDevice(s->device));
    return s->set.precision == MFS_FP64 ? s_warm(s, s->f64, x, lambda) : s_warm(s, s->f32, x, lambda);
}

mfs_status mfs_shared_iterate(mfs_shared* s, int64_t k) {
    MFS_TRACE("mfs_shared_iterate");
    if (!s || k < 0) return MFS_ERR_INVALID;
    SCUDA(s, cudaSetDevice(s->device));
    STRY(s->set.precision == MFS_FP64 ? s_run(s, s->f64, k) : s_run(s, s->f32, k));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_shared_residuals(mfs_shared* s, mfs_residuals_t* out) {
    if (!s || !out) return MFS_ERR_INVALID;
    SCUDA(s, cudaSetDevice(s->device));
    if (s->set.precision == MFS_FP64) {
        STRY(s_residuals(s, s->f64, (double*)nullptr));
    } else {
        STRY(s_residuals(s, s->f32, (float*)nullptr));
    }
    SCUDA(s, cudaMemcpyAsync(s->h_status, s->status, (size_t)NSTAT * s->B * sizeof(double), cudaMemcpyDeviceToHost,
                             s->stream));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    for (int t = 0; t < s->B; ++t) {
        double* d = reinterpret_cast<double*>(&out[t]);
        for (int q = 0; q < NSTAT; ++q) d[q] = s->h_status[(size_t)t * NSTAT + q];
        mfs::stop_measures(&out[t], s->set.osqp_rel);
        out[t].iter = s->iter;
    }
    return MFS_OK;
}

/* Iterate all instances, testing each every check_every iterations, until every instance's
   relative KKT residual is <= tol or max_iter iterations have run; iters[t] (nullable) receives
   the iteration at which instance t first met tol, or -1. Returns MFS_OK if all met it. */
mfs_status mfs_shared_solve(mfs_shared* s, double tol, int64_t max_iter, int64_t* iters) {
    MFS_TRACE("mfs_shared_solve");
    if (!s || !(tol > 0.0) || max_iter < 0) return MFS_ERR_INVALID;
    std::vector<int64_t> first(s->B, -1);
    std::vector<mfs_residuals_t> r(s->B);
    const int64_t K = std::max(1, (int)s->set.check_every);
    int64_t it = 0;
    int remaining = s->B;
    for (;;) {
        STRY(mfs_shared_residuals(s, r.data()));
        for (int t = 0; t < s->B; ++t) {
            if (!std::isfinite(r[t].kkt)) return sfail(s, MFS_ERR_NUMERIC, "NaN or Inf in the residuals");
            if (first[t] < 0 && r[t].kkt <= tol) {
                first[t] = it;
                --remaining;
            }
        }
        if (remaining == 0 || it >= max_iter) break;
        const int64_t kk = std::min<int64_t>(K, max_iter - it);
        STRY(mfs_shared_iterate(s, kk));
        it += kk;
    }
    if (iters)
        for (int t = 0; t < s->B; ++t) iters[t] = first[t];
    return remaining == 0 ? MFS_OK : MFS_MAX_ITER;
}

/* iterate in instance-major layout on the device: x [count][n], lambda [count][m] (FP32) */
mfs_status mfs_shared_get_solution_device(mfs_shared* s, float* x, float* lambda) {
    if (!s) return MFS_ERR_INVALID;
    SCUDA(s, cudaSetDevice(s->device));
    if (s->set.precision == MFS_FP64) {
        if (x) deinterleave(s->f64.x, x, s->B, s->n, s->Bp, s->stream);
        if (lambda) deinterleave(s->f64.lam, lambda, s->B, s->m, s->Bp, s->stream);
    } else {
        if (x) deinterleave(s->f32.x, x, s->B, s->n, s->Bp, s->stream);
        if (lambda) deinterleave(s->f32.lam, lambda, s->B, s->m, s->Bp, s->stream);
    }
    SCUDA(s, cudaGetLastError());
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_shared_load_slots_warm(mfs_shared* s, int64_t count, const int32_t* slots, const float* b,
                                      const float* c, const float* x, const float* lambda) {
    if (!s) return MFS_ERR_INVALID;
    if (count > 0 && ((s->m && (!b || !lambda)) || (s->n && (!c || !x))))
        return sfail(s, MFS_ERR_INVALID, "b, c, x and lambda are required");
    STRY(mfs_shared_load_slots(s, count, slots, b, c));
    if (count)
        STRY(s->set.precision == MFS_FP64 ? warm_slots_t(s, s->f64, (int)count, x, lambda)
                                          : warm_slots_t(s, s->f32, (int)count, x, lambda));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_shared_load_slots(mfs_shared* s, int64_t count, const int32_t* slots, const float* b, const float* c) {
    if (!s) return MFS_ERR_INVALID;
    if (count > 0 && ((s->m && !b) || (s->n && !c))) return sfail(s, MFS_ERR_INVALID, "b and c are required");
    SCUDA(s, cudaSetDevice(s->device));
    STRY(put_slots(s, count, slots));
    if (count)
        STRY(s->set.precision == MFS_FP64 ? load_slots_t(s, s->f64, (int)count, b, c)
                                          : load_slots_t(s, s->f32, (int)count, b, c));
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_shared_get_slots_device(mfs_shared* s, int64_t count, const int32_t* slots, float* x, float* lambda) {
    if (!s) return MFS_ERR_INVALID;
    SCUDA(s, cudaSetDevice(s->device));
    STRY(put_slots(s, count, slots));
    const long long tm = count * (long long)s->m, tn = count * (long long)s->n;
    if (s->set.precision == MFS_FP64) {
        if (x && tn) k_s_gather_slots<double, float><<<grid_for(tn), 256, 0, s->stream>>>(s->f64.x, x, s->slot_buf, (int)count, s->n, s->Bp);
        if (lambda && tm) k_s_gather_slots<double, float><<<grid_for(tm), 256, 0, s->stream>>>(s->f64.lam, lambda, s->slot_buf, (int)count, s->m, s->Bp);
    } else {
        if (x && tn) k_s_gather_slots<float, float><<<grid_for(tn), 256, 0, s->stream>>>(s->f32.x, x, s->slot_buf, (int)count, s->n, s->Bp);
        if (lambda && tm) k_s_gather_slots<float, float><<<grid_for(tm), 256, 0, s->stream>>>(s->f32.lam, lambda, s->slot_buf, (int)count, s->m, s->Bp);
    }
    SCUDA(s, cudaGetLastError());
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

/* iterate of instance t as host doubles (any pointer may be NULL) */
mfs_status mfs_shared_get_solution(mfs_shared* s, int64_t t, double* x, double* lambda, double* z, double* delta) {
    if (!s || t < 0 || t >= s->B) return MFS_ERR_INVALID;
    SCUDA(s, cudaSetDevice(s->device));
    double* tmp = nullptr;
    const size_t nb = (size_t)s->n, mb = (size_t)s->m;
    SCUDA(s, cudaMallocAsync((void**)&tmp, std::max<size_t>(1, 3 * nb + mb) * sizeof(double), s->stream));
    auto one = [&](auto* src, int len, double* dev, double* host) {
        if (!host || !len) return;
        k_s_extract<<<std::min((len + 255) / 256, 1024), 256, 0, s->stream>>>(src, dev, len, s->Bp, (int)t);
        cudaMemcpyAsync(host, dev, len * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    };
    if (s->set.precision == MFS_FP64) {
        one(s->f64.x, s->n, tmp, x);
        one(s->f64.lam, s->m, tmp + nb, lambda);
        one(s->f64.z, s->n, tmp + nb + mb, z);
        one(s->f64.del, s->n, tmp + 2 * nb + mb, delta);
    } else {
        one(s->f32.x, s->n, tmp, x);
        one(s->f32.lam, s->m, tmp + nb, lambda);
        one(s->f32.z, s->n, tmp + nb + mb, z);
        one(s->f32.del, s->n, tmp + 2 * nb + mb, delta);
    }
    cudaFreeAsync(tmp, s->stream);
    SCUDA(s, cudaGetLastError());
    SCUDA(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

}  // extern "C"
