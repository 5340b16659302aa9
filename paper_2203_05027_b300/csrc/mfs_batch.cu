// mfs_batch.cu -- batched solves: thousands of independent conic programs of uneven sizes in one
// persistent launch (the mfs_batch_* calls of include/mfs.h).
//
// Each CTA takes instances from an atomic queue (largest first) and runs Algorithm 1 on one
// instance at a time, in the reduced form of the single-instance solver (column sweep with the
// x-step, z-step and delta-update; row sweep with the y-step and lambda-update), with
// __syncthreads between the two sweeps. The two vectors the sweeps gather from (x in the row
// sweep, v = F_U (b - A x) - lambda/mu in the column sweep) are held in shared memory for the
// whole run of an instance, so the per-nonzero gathers never leave the SM; the instance's matrix
// (both orders) is cached in shared memory as well when it fits, otherwise streamed from global
// memory. Residuals are reduced in FP64 inside the CTA every check_every iterations when a
// tolerance is given, and an instance stops as soon as it meets it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/mfs.h"
#include "mfs_trace.h"
#include "mfs_alloc.h"
#include "mfs_device.cuh"
#include "mfs_host.h"
#include "mfs_measures.h"

namespace {

using mfs::DF;
using mfs::FULL;

constexpr int MAXNT = 512;
constexpr int MAXW = MAXNT / 32;
constexpr int FVT = 64;  // column lengths with a tabulated F_V
constexpr int NSTAT = 23;  // status block, same order as mfs_residuals_t

template <typename T>
struct BatchArgs {
    int count;
    const int* order;  // processing order (largest first)
    const int* m;
    const int* n;
    const int* o;
    const long long* off_n;  // first coordinate of each instance in the n-length arrays
    const long long* off_m;
    const long long* off_o;  // first nonzero of each instance
    const int* col_ptr;      // instance t: n[t]+1 local offsets starting at off_n[t] + t
    const int* cidx;         // local row indices, column order
    const T* cval;
    const int* row_ptr;      // instance t: m[t]+1 local offsets starting at off_m[t] + t
    const int* ridx;         // local column indices, row order
    const uint16_t* cidx16;  // the same as 16-bit indices, when every instance has m, n <= 65535
    const uint16_t* ridx16;  // (then cidx and ridx are not stored)
    const T* rval;
    const T* fu;             // F_U = 1 / (1 + sum_k a_ik^2) per row
    const int* nsoc;         // Lorentz cones per instance (local starts, ascending)
    const long long* off_soc;
    const int* soc_start;
    const int* soc_size;
    const T* b;
    const T* c;
    T* x;
    T* z;
    T* del;
    T* lam;
    T* v;
    T mu;
    int iters;        // iterations for each instance in this launch (at most, when tol > 0)
    double tol;       // > 0: an instance stops once its relative KKT residual is <= tol
    int check_every;  // iterations between residual checks
    int smem_bytes;   // dynamic shared memory of a CTA
    int* queue;       // instance counter, zero at launch
    long long* iters_done;
    int* status;      // 0 = met tol, 1 = not (yet)
    double* resid;    // NSTAT doubles per instance, last evaluation
};

template <typename T>
struct AccT {
    using type = DF;
};
template <>
struct AccT<double> {
    using type = double;
};
__device__ __forceinline__ DF acc_mul(float a, float b) { return mfs::df_prod(a, b); }
__device__ __forceinline__ double acc_mul(double a, double b) { return a * b; }


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

// sum over k in [k0, k1) of val[k] * vec[idx[k]], added in order of k: the loads of up to four
// entries are issued together (a column or row of A read from memory is otherwise a chain of
// dependent round trips, one per nonzero), the products added one after another as before
#ifndef MFS_BATCH_SEG_UNROLL
#define MFS_BATCH_SEG_UNROLL 4
#endif
template <typename T, typename IT>
__device__ __forceinline__ T seg_dot(const IT* idx, const T* val, int k0, int k1, const T* vec) {
    constexpr int U = MFS_BATCH_SEG_UNROLL;
    T s = T(0);
    for (int k = k0; k < k1; k += U) {
        int ix[U];
        T av[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool in = k + u < k1;
            ix[u] = in ? idx[k + u] : 0;
            av[u] = in ? val[k + u] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (k + u < k1) s += av[u] * vec[ix[u]];
    }
    return s;
}

// the Lorentz cone (local index) that contains column j, or -1
__device__ __forceinline__ int cone_of(const int* st, const int* sz, int ns, int j) {
    int lo = 0, hi = ns;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (st[mid] <= j)
            lo = mid + 1;
        else
            hi = mid;
    }
    const int q = lo - 1;
    return (q >= 0 && j < st[q] + sz[q]) ? q : -1;
}

// Block-wide fold of NF doubles (fields flagged in maxmask are maxima); result in thread 0.
template <int NF>
__device__ __forceinline__ void block_fold(double (&f)[NF], unsigned maxmask, double (*sh)[NF]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        double v = f[k];
        for (int d = 16; d > 0; d >>= 1) {
            const double o = __shfl_down_sync(FULL, v, d);
            v = ((maxmask >> k) & 1u) ? fmax(v, o) : v + o;
        }
        f[k] = v;
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NF; ++k) sh[warp][k] = f[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            double acc = 0.0;
            for (int w = 0; w < nw; ++w) acc = ((maxmask >> k) & 1u) ? fmax(acc, sh[w][k]) : acc + sh[w][k];
            f[k] = acc;
        }
    }
}

// Block-wide fold of NF double-float pairs in FP32 arithmetic (fields flagged in maxmask are maxima);
// result in thread 0. A warp-wide FP64 shuffle fold occupies the SM's narrow FP64 pipe for every
// field and round, which made the FP64 fold half of a residual check's time.
template <int NF>
__device__ __forceinline__ void block_fold_df(DF (&F)[NF], unsigned maxmask, DF (*sh)[NF]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NF; ++k) {
        DF v = F[k];
        for (int d = 16; d > 0; d >>= 1) {
            const DF o(__shfl_down_sync(FULL, v.hi, d), __shfl_down_sync(FULL, v.lo, d));
            v = ((maxmask >> k) & 1u) ? mfs::df_max(v, o) : v + o;
        }
        F[k] = v;
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NF; ++k) sh[warp][k] = F[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NF; ++k) {
            DF v = lane < nw ? sh[lane][k] : DF(0);
            for (int d = 16; d > 0; d >>= 1) {
                const DF o(__shfl_down_sync(FULL, v.hi, d), __shfl_down_sync(FULL, v.lo, d));
                v = ((maxmask >> k) & 1u) ? mfs::df_max(v, o) : v + o;
            }
            F[k] = v;
        }
    }
}

// fields of the residual fold
enum { RES2, RESMAX, AXMAX, B2, BMAX, BLAM, S2, SMAX, ATLMAX, C2, CMAX, CX, X2, SDIST2, XDIST2, XMAX, SDMAX, XDMAX, NFLD };
constexpr unsigned MAXMASK = (1u << RESMAX) | (1u << AXMAX) | (1u << BMAX) | (1u << SMAX) | (1u << ATLMAX) | (1u << CMAX) |
                           (1u << XMAX) | (1u << SDMAX) | (1u << XDMAX);

struct Inst {
    int t, m, n, o, ns;
    long long gn, gm, go, gs;
};

// FP64 residuals of instance I at (x, lambda) (x read through xs); status block into out[NSTAT]
// (thread 0) and the relative KKT residual returned to every thread. For the FP32 iterate the row
// and column fields are kept, and folded over the block, as double-float pairs (about 48
// significant bits) and turned into FP64 by thread 0 only (B300 runs FP64 at 1/64 of its FP32
// rate); the Lorentz cones' terms are formed in FP64 and added as pairs.
template <typename T, typename IT>
__device__ double instance_residuals(const BatchArgs<T>& a, const Inst& I, const T* xs, const T* lam, const int* cp,
                                     const IT* ci,
                                     const T* cv, const int* rp, const IT* ri, const T* rv, double* out,
                                     double (*sh)[NFLD], double* s_kkt) {
    using A = typename AccT<T>::type;
    constexpr bool F32 = std::is_same<T, float>::value;
    double f[NFLD];
#pragma unroll
    for (int k = 0; k < NFLD; ++k) f[k] = 0.0;
    DF F[F32 ? NFLD : 1];
#pragma unroll
    for (int k = 0; k < (F32 ? NFLD : 1); ++k) F[k] = DF(0);
    for (int i = threadIdx.x; i < I.m; i += blockDim.x) {
        A acc = A(0);
        for (int k = rp[i]; k < rp[i + 1]; ++k) acc = acc + acc_mul(rv[k], xs[ri[k]]);
        if constexpr (F32) {
            const float bi = a.b[I.gm + i];
            const DF res = acc + DF(-bi, 0.f);
            F[RES2] = F[RES2] + mfs::df_sq(res);
            F[RESMAX] = mfs::df_max(F[RESMAX], mfs::df_abs(res));
            F[AXMAX] = mfs::df_max(F[AXMAX], mfs::df_abs(acc));
            F[B2] = F[B2] + mfs::df_prod(bi, bi);
            F[BMAX] = mfs::df_max(F[BMAX], DF(fabsf(bi), 0.f));
            F[BLAM] = F[BLAM] + mfs::df_prod(bi, lam[i]);
            continue;
        }
        const double ax = mfs::to_double(acc), bi = double(a.b[I.gm + i]), res = ax - bi;
        f[RES2] += res * res;
        f[RESMAX] = fmax(f[RESMAX], fabs(res));
        f[AXMAX] = fmax(f[AXMAX], fabs(ax));
        f[B2] += bi * bi;
        f[BMAX] = fmax(f[BMAX], fabs(bi));
        f[BLAM] += bi * double(lam[i]);
    }
    const int* sst = a.soc_start + I.gs;
    const int* ssz = a.soc_size + I.gs;
    auto column = [&](int j, bool orthant, double& s_out) {
        A acc = A(0);
        for (int k = cp[j]; k < cp[j + 1]; ++k) acc = acc + acc_mul(cv[k], lam[ci[k]]);
        if constexpr (F32) {
            const float cj = a.c[I.gn + j], xj = xs[j];
            const DF sd = DF(cj, 0.f) + acc;
            F[S2] = F[S2] + mfs::df_sq(sd);
            F[SMAX] = mfs::df_max(F[SMAX], mfs::df_abs(sd));
            F[ATLMAX] = mfs::df_max(F[ATLMAX], mfs::df_abs(acc));
            F[C2] = F[C2] + mfs::df_prod(cj, cj);
            F[CMAX] = mfs::df_max(F[CMAX], DF(fabsf(cj), 0.f));
            F[CX] = F[CX] + mfs::df_prod(cj, xj);
            F[X2] = F[X2] + mfs::df_prod(xj, xj);
            F[XMAX] = mfs::df_max(F[XMAX], DF(fabsf(xj), 0.f));
            if (orthant) {
                const DF sn = sd.hi < 0.f ? sd : DF(0);
                const float xn = xj < 0.f ? xj : 0.f;
                F[SDIST2] = F[SDIST2] + mfs::df_sq(sn);
                F[XDIST2] = F[XDIST2] + mfs::df_prod(xn, xn);
                F[SDMAX] = mfs::df_max(F[SDMAX], mfs::df_neg(sn));
                F[XDMAX] = mfs::df_max(F[XDMAX], DF(-xn, 0.f));
                s_out = 0.0;
            } else {
                s_out = mfs::to_double(sd);
            }
            return;
        }
        const double atl = mfs::to_double(acc), cj = double(a.c[I.gn + j]), xj = double(xs[j]);
        const double s = cj + atl;
        f[S2] += s * s;
        f[SMAX] = fmax(f[SMAX], fabs(s));
        f[ATLMAX] = fmax(f[ATLMAX], fabs(atl));
        f[C2] += cj * cj;
        f[CMAX] = fmax(f[CMAX], fabs(cj));
        f[CX] += cj * xj;
        f[X2] += xj * xj;
        f[XMAX] = fmax(f[XMAX], fabs(xj));
        if (orthant) {
            const double sn = s < 0.0 ? s : 0.0, xn = xj < 0.0 ? xj : 0.0;
            f[SDIST2] += sn * sn;
            f[XDIST2] += xn * xn;
            f[SDMAX] = fmax(f[SDMAX], -sn);
            f[XDMAX] = fmax(f[XDMAX], -xn);
        }
        s_out = s;
    };
    for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
        if (I.ns && cone_of(sst, ssz, I.ns, j) >= 0) continue;
        double s;
        column(j, true, s);
    }
    for (int q = threadIdx.x; q < I.ns; q += blockDim.x) {  // one thread per Lorentz cone
        double s1 = 0.0, ss = 0.0, x1 = 0.0, xx = 0.0;
        for (int t = 0; t < ssz[q]; ++t) {
            const int j = sst[q] + t;
            double s;
            column(j, false, s);
            const double xj = double(xs[j]);
            if (t == 0) {
                s1 = s;
                x1 = xj;
            } else {
                ss += s * s;
                xx += xj * xj;
            }
        }
        if constexpr (F32) {
            F[SDIST2] = F[SDIST2] + mfs::df_from(lorentz_dist2(s1, sqrt(ss), ss + s1 * s1));
            F[XDIST2] = F[XDIST2] + mfs::df_from(lorentz_dist2(x1, sqrt(xx), xx + x1 * x1));
            F[SDMAX] = mfs::df_max(F[SDMAX], mfs::df_from(mfs::lorentz_distinf(s1, sqrt(ss))));
            F[XDMAX] = mfs::df_max(F[XDMAX], mfs::df_from(mfs::lorentz_distinf(x1, sqrt(xx))));
        } else {
            f[SDIST2] += lorentz_dist2(s1, sqrt(ss), ss + s1 * s1);
            f[XDIST2] += lorentz_dist2(x1, sqrt(xx), xx + x1 * x1);
            f[SDMAX] = fmax(f[SDMAX], mfs::lorentz_distinf(s1, sqrt(ss)));
            f[XDMAX] = fmax(f[XDMAX], mfs::lorentz_distinf(x1, sqrt(xx)));
        }
    }
    if constexpr (F32) {
        block_fold_df<NFLD>(F, MAXMASK, reinterpret_cast<DF(*)[NFLD]>(sh));
        if (threadIdx.x == 0)
#pragma unroll
            for (int k = 0; k < NFLD; ++k) f[k] = mfs::to_double(F[k]);
    } else {
        block_fold<NFLD>(f, MAXMASK, sh);
    }
    if (threadIdx.x == 0) {
        const double nres = sqrt(f[RES2]), nb = sqrt(f[B2]), nxd = sqrt(f[XDIST2]), nx = sqrt(f[X2]);
        const double nsd = sqrt(f[SDIST2]), nc = sqrt(f[C2]), cx = f[CX], bl = f[BLAM];
        double st[NSTAT];
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
        for (int q = 0; q < NSTAT; ++q) out[q] = st[q];
        *s_kkt = kkt;
    }
    __syncthreads();
    return *s_kkt;
}

template <typename T>
__device__ __forceinline__ Inst load_inst(const BatchArgs<T>& a, int t) {
    Inst I;
    I.t = t;
    I.m = a.m[t];
    I.n = a.n[t];
    I.o = a.o[t];
    I.ns = a.nsoc[t];
    I.gn = a.off_n[t];
    I.gm = a.off_m[t];
    I.go = a.off_o[t];
    I.gs = a.off_soc[t];
    return I;
}

// MODE 0: iterate with termination checks (tol > 0); MODE 1: residuals only; MODE 2: iterate
// without checks (tol = 0; no residual code in the kernel, so none of its registers either).
#ifndef MFS_BATCH_MINB
#define MFS_BATCH_MINB 2  // 64 registers: two 512-thread CTAs per SM
#endif

// the index arrays of the width IT
template <typename IT>
__device__ __forceinline__ const IT* idx_of(const int* i32, const uint16_t* i16) {
    if constexpr (sizeof(IT) == 2)
        return i16;
    else
        return i32;
}

template <typename T, typename IT, int MODE>
__global__ void __launch_bounds__(MAXNT, MFS_BATCH_MINB) k_batch(const BatchArgs<T> a) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double s_red[MAXW][NFLD];
    __shared__ double s_kkt;
    __shared__ int s_inst;
    __shared__ T s_fv[FVT];  // F_V = 1 / (1 + d) for column lengths d < FVT
    const T mu = a.mu, inv_mu = T(1) / a.mu;
    for (int d = threadIdx.x; d < FVT; d += blockDim.x) s_fv[d] = T(1) / (T(1) + T(d));
    for (;;) {
        if (threadIdx.x == 0) s_inst = atomicAdd(a.queue, 1);
        __syncthreads();
        const int q = s_inst;
        __syncthreads();
        if (q >= a.count) break;
        const Inst I = load_inst(a, a.order[q]);
        // shared memory: gathered vectors first, then (if room) the matrix in both orders
        const size_t vb = (size_t)(I.n + I.m) * sizeof(T);
        const size_t ab = (size_t)I.o * 2 * (sizeof(IT) + sizeof(T));
        const bool vec_sm = vb <= (size_t)a.smem_bytes;
        const bool mat_sm = vec_sm && (vb + ab + 16 <= (size_t)a.smem_bytes);
        T* xs = vec_sm ? reinterpret_cast<T*>(sm) : a.x + I.gn;
        T* vs = vec_sm ? reinterpret_cast<T*>(sm) + I.n : a.v + I.gm;
        const int* cp = a.col_ptr + I.gn + I.t;
        const int* rp = a.row_ptr + I.gm + I.t;
        const IT* ci = idx_of<IT>(a.cidx, a.cidx16) + I.go;
        const T* cv = a.cval + I.go;
        const IT* ri = idx_of<IT>(a.ridx, a.ridx16) + I.go;
        const T* rv = a.rval + I.go;
        if (vec_sm) {
            for (int j = threadIdx.x; j < I.n; j += blockDim.x) xs[j] = a.x[I.gn + j];
            for (int i = threadIdx.x; i < I.m; i += blockDim.x) vs[i] = a.v[I.gm + i];
        }
        if (mat_sm) {
            unsigned char* p = sm + ((vb + 15) & ~size_t(15));
            T* scv = reinterpret_cast<T*>(p);
            T* srv = scv + I.o;
            IT* sci = reinterpret_cast<IT*>(srv + I.o);
            IT* sri = sci + I.o;
            for (int k = threadIdx.x; k < I.o; k += blockDim.x) {
                scv[k] = cv[k];
                srv[k] = rv[k];
                sci[k] = ci[k];
                sri[k] = ri[k];
            }
            cv = scv;
            rv = srv;
            ci = sci;
            ri = sri;
        }
        __syncthreads();
        const int* sst = a.soc_start + I.gs;
        const int* ssz = a.soc_size + I.gs;
        T* z = a.z + I.gn;
        T* del = a.del + I.gn;
        const T* c = a.c + I.gn;
        const T* b = a.b + I.gm;
        const T* fu = a.fu + I.gm;
        T* lam = a.lam + I.gm;
        int done = 0;
        int met = 0;
        if (MODE != 1) {
            for (; done < a.iters;) {
                // column sweep: x-step (eq. vvt), z-step and delta-update for orthant coordinates
                for (int j = threadIdx.x; j < I.n; j += blockDim.x) {
                    const int k0 = cp[j], k1 = cp[j + 1];
                    const T s = seg_dot(ci, cv, k0, k1, vs);
                    const T d = T(k1 - k0), dj = del[j];
                    const T fv = k1 - k0 < FVT ? s_fv[k1 - k0] : T(1) / (T(1) + d);
                    const T xn = (d * xs[j] + s + z[j] + (dj - c[j]) * inv_mu) * fv;
                    xs[j] = xn;
                    if (I.ns == 0 || cone_of(sst, ssz, I.ns, j) < 0) {
                        const T w = xn - dj * inv_mu;
                        const T zn = w > T(0) ? w : T(0);
                        z[j] = zn;
                        del[j] = dj + mu * (zn - xn);
                    }
                }
                __syncthreads();
                if (I.ns) {  // z-step (eq. proj) and delta-update of the Lorentz cones, one thread each
                    for (int qc = threadIdx.x; qc < I.ns; qc += blockDim.x) {
                        const int s0 = sst[qc], sz = ssz[qc];
                        T ss = T(0);
                        for (int t = 1; t < sz; ++t) {
                            const T w = xs[s0 + t] - del[s0 + t] * inv_mu;
                            ss += w * w;
                        }
                        const T alpha = sqrt(ss), w1 = xs[s0] - del[s0] * inv_mu;
                        for (int t = 0; t < sz; ++t) {
                            const T xt = xs[s0 + t], dt = del[s0 + t];
                            const T zt = lorentz_coord(xt - dt * inv_mu, t, w1, alpha);
                            z[s0 + t] = zt;
                            del[s0 + t] = dt + mu * (zt - xt);
                        }
                    }
                    __syncthreads();
                }
                // row sweep: y-step (with F_U) and lambda-update
                for (int i = threadIdx.x; i < I.m; i += blockDim.x) {
                    const T s = seg_dot(ri, rv, rp[i], rp[i + 1], xs);
                    const T rho = (b[i] - s) * fu[i];
                    const T ln = lam[i] - mu * rho;
                    lam[i] = ln;
                    vs[i] = rho - ln * inv_mu;
                }
                __syncthreads();
                ++done;
                if (MODE == 0 && a.tol > 0.0 && (done % a.check_every == 0 || done == a.iters)) {
                    const double kkt = instance_residuals(a, I, xs, lam, cp, ci, cv, rp, ri, rv,
                                                          a.resid + (size_t)I.t * NSTAT, s_red, &s_kkt);
                    if (kkt <= a.tol) {
                        met = 1;
                        break;
                    }
                }
            }
        } else {
            instance_residuals(a, I, xs, lam, cp, ci, cv, rp, ri, rv, a.resid + (size_t)I.t * NSTAT, s_red,
                               &s_kkt);
        }
        __syncthreads();
        if (vec_sm && MODE != 1) {
            for (int j = threadIdx.x; j < I.n; j += blockDim.x) a.x[I.gn + j] = xs[j];
            for (int i = threadIdx.x; i < I.m; i += blockDim.x) a.v[I.gm + i] = vs[i];
        }
        if (threadIdx.x == 0 && MODE != 1) {
            a.iters_done[I.t] += done;
            a.status[I.t] = met ? 0 : 1;
        }
        __syncthreads();
    }
}

template <typename T>
struct Store {
    T *cval = nullptr, *rval = nullptr, *fu = nullptr, *b = nullptr, *c = nullptr;
    T *x = nullptr, *z = nullptr, *del = nullptr, *lam = nullptr, *v = nullptr;
};

}  // namespace

struct mfs_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    mfs_settings set{};
    mfs_batch_tuning tune{};
    int count = 0;
    int64_t tot_n = 0, tot_m = 0, tot_o = 0, tot_soc = 0;
    int max_smem = 0, max_smem_block = 0, num_sms = 148;
    int static_smem = 0;  // largest static shared memory of the k_batch instantiations
    std::vector<int> hm, hn, ho;
    std::vector<long long> hoff_n, hoff_m, hoff_o;
    int *order = nullptr, *m = nullptr, *n = nullptr, *o = nullptr, *nsoc = nullptr;
    long long *off_n = nullptr, *off_m = nullptr, *off_o = nullptr, *off_soc = nullptr;
    int *col_ptr = nullptr, *cidx = nullptr, *row_ptr = nullptr, *ridx = nullptr;
    bool idx16 = false;  // every instance has m, n <= 65535: 16-bit local indices
    uint16_t *cidx16 = nullptr, *ridx16 = nullptr;
    int *soc_start = nullptr, *soc_size = nullptr;
    int* queue = nullptr;
    long long* iters_done = nullptr;
    int* status = nullptr;
    double* resid = nullptr;
    Store<float> f32;
    Store<double> f64;
    cudaGraphExec_t graph = nullptr;
    int graph_iters = -1;
    double graph_tol = -1;
    std::vector<void*> allocs;
    std::string last_error;
};

namespace {

thread_local std::string g_batch_create_error;

mfs_status bfail(mfs_batch* s, mfs_status st, const std::string& msg) {
    if (s)
        s->last_error = msg;
    else
        g_batch_create_error = msg;
    return st;
}

#define BCUDA(s, call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bfail((s), e_ == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA,         \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)
#define BTRY(x)                         \
    do {                                \
        mfs_status st_ = (x);           \
        if (st_ != MFS_OK) return st_;  \
    } while (0)

template <typename T>
mfs_status bupload(mfs_batch* s, T** p, const void* host, size_t count) {
    void* q = nullptr;
    BCUDA(s, mfs::device_malloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
    s->allocs.push_back(q);
    *p = static_cast<T*>(q);
    if (count) BCUDA(s, cudaMemcpyAsync(q, host, count * sizeof(T), cudaMemcpyHostToDevice, s->stream));
    return MFS_OK;
}

template <typename T>
mfs_status bzeros(mfs_batch* s, T** p, size_t count) {
    void* q = nullptr;
    BCUDA(s, mfs::device_malloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
    s->allocs.push_back(q);
    *p = static_cast<T*>(q);
    BCUDA(s, cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), s->stream));
    return MFS_OK;
}

template <typename T>
BatchArgs<T> batch_args(mfs_batch* s, Store<T>& st, int iters, double tol) {
    BatchArgs<T> a;
    a.count = s->count;
    a.order = s->order;
    a.m = s->m;
    a.n = s->n;
    a.o = s->o;
    a.off_n = s->off_n;
    a.off_m = s->off_m;
    a.off_o = s->off_o;
    a.col_ptr = s->col_ptr;
    a.cidx = s->cidx;
    a.cval = st.cval;
    a.row_ptr = s->row_ptr;
    a.ridx = s->ridx;
    a.cidx16 = s->cidx16;
    a.ridx16 = s->ridx16;
    a.rval = st.rval;
    a.fu = st.fu;
    a.nsoc = s->nsoc;
    a.off_soc = s->off_soc;
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
    a.iters = iters;
    a.tol = tol;
    a.check_every = std::max(1, (int)s->set.check_every);
    a.smem_bytes = 0;
    a.queue = s->queue;
    a.iters_done = s->iters_done;
    a.status = s->status;
    a.resid = s->resid;
    return a;
}

// Dynamic shared memory per CTA for the current tuning (ctas_per_sm CTAs share an SM).
int smem_for(const mfs_batch* s) {
    const int per = s->max_smem / std::max(1, (int)s->tune.ctas_per_sm);
    const int stat = s->static_smem + 64;
    return std::max(0, std::min(per - stat - 1024, s->max_smem_block - stat));
}

template <typename T, int MODE>
mfs_status launch_batch(mfs_batch* s, Store<T>& st, int iters, double tol, cudaStream_t stream) {
    BatchArgs<T> a = batch_args(s, st, iters, tol);
    a.smem_bytes = smem_for(s);
    auto kern = s->idx16 ? k_batch<T, uint16_t, MODE> : k_batch<T, int, MODE>;
    BCUDA(s, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes));
    BCUDA(s, cudaMemsetAsync(s->queue, 0, sizeof(int), stream));
    const int grid = std::max(1, std::min(s->count, s->num_sms * std::max(1, (int)s->tune.ctas_per_sm)));
    kern<<<grid, s->tune.threads, a.smem_bytes, stream>>>(a);
    BCUDA(s, cudaGetLastError());
    return MFS_OK;
}

template <typename T>
mfs_status run_batch(mfs_batch* s, Store<T>& st, int iters, double tol) {
    // the persistent launch (queue reset + kernel) is captured once per (iters, tol) and replayed
    if (!s->graph || s->graph_iters != iters || s->graph_tol != tol) {
        if (s->graph) cudaGraphExecDestroy(s->graph);
        s->graph = nullptr;
        cudaStream_t cap = nullptr;
        BCUDA(s, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        mfs_status ms = MFS_OK;
        if (e == cudaSuccess) {
            ms = tol > 0.0 ? launch_batch<T, 0>(s, st, iters, tol, cap) : launch_batch<T, 2>(s, st, iters, tol, cap);
            e = cudaStreamEndCapture(cap, &g);
        }
        if (e == cudaSuccess && ms == MFS_OK) e = cudaGraphInstantiate(&s->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
        if (ms != MFS_OK) return ms;
        if (e != cudaSuccess) {
            s->graph = nullptr;
            return bfail(s, MFS_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        }
        s->graph_iters = iters;
        s->graph_tol = tol;
    }
    BCUDA(s, cudaGraphLaunch(s->graph, s->stream));
    BCUDA(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

template <typename T>
mfs_status alloc_store(mfs_batch* s, Store<T>& st, const std::vector<double>& cval, const std::vector<double>& rval,
                       const std::vector<int>& rp, const double* b, const double* c) {
    std::vector<T> tmp(cval.begin(), cval.end());
    BTRY(bupload(s, &st.cval, tmp.data(), tmp.size()));
    tmp.assign(rval.begin(), rval.end());
    BTRY(bupload(s, &st.rval, tmp.data(), tmp.size()));
    // F_U from the stored (T-rounded) values, summed in FP64: per instance t, rows i take the
    // nonzeros rp[off_m + t + i] .. rp[off_m + t + i + 1] of that instance's row order
    std::vector<T> fu(s->tot_m);
    for (int t = 0; t < s->count; ++t) {
        const long long rb = s->hoff_m[t] + t, ob = s->hoff_o[t];
        for (int i = 0; i < s->hm[t]; ++i) {
            double r = 0.0;
            for (int k = rp[rb + i]; k < rp[rb + i + 1]; ++k) {
                const double a = double(tmp[ob + k]);
                r += a * a;
            }
            fu[s->hoff_m[t] + i] = T(1.0 / (1.0 + r));
        }
    }
    BTRY(bupload(s, &st.fu, fu.data(), fu.size()));
    tmp.assign(b, b + s->tot_m);
    BTRY(bupload(s, &st.b, tmp.data(), tmp.size()));
    tmp.assign(c, c + s->tot_n);
    BTRY(bupload(s, &st.c, tmp.data(), tmp.size()));
    BTRY(bzeros(s, &st.x, s->tot_n));
    BTRY(bzeros(s, &st.z, s->tot_n));
    BTRY(bzeros(s, &st.del, s->tot_n));
    BTRY(bzeros(s, &st.lam, s->tot_m));
    BTRY(bzeros(s, &st.v, s->tot_m));
    return MFS_OK;
}

template <typename T>
__global__ void k_to_double(double* dst, const T* src, long long count) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x)
        dst[t] = double(src[t]);
}

}  // namespace

extern "C" {

mfs_status mfs_batch_create(int64_t count, const int64_t* m, const int64_t* n, const int64_t* nnz, const int64_t* row,
                            const int64_t* col, const double* val, const double* b, const double* c,
                            const int64_t* ncones, const mfs_cone* cones, const mfs_settings* settings,
                            void* cuda_stream, mfs_batch** out) {
    MFS_TRACE("mfs_batch_create");
    g_batch_create_error.clear();
    if (!out) return bfail(nullptr, MFS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (count < 1 || !m || !n || !nnz || !ncones) return bfail(nullptr, MFS_ERR_INVALID, "count < 1 or NULL sizes");
    mfs_settings set;
    mfs_default_settings(&set);
    if (settings) set = *settings;
    if (!(set.mu > 0.0) || !std::isfinite(set.mu) || set.check_every < 1 ||
        (set.precision != MFS_FP64 && set.precision != MFS_FP32_MIXED))
        return bfail(nullptr, MFS_ERR_INVALID, "invalid settings");
    int64_t tn = 0, tm = 0, to = 0, tc = 0;
    for (int64_t t = 0; t < count; ++t) {
        if (m[t] < 0 || n[t] < 0 || nnz[t] < 0 || ncones[t] < 0 || m[t] >= INT32_MAX || n[t] >= INT32_MAX)
            return bfail(nullptr, MFS_ERR_INVALID, "bad sizes of instance " + std::to_string(t));
        tn += n[t];
        tm += m[t];
        to += nnz[t];
        tc += ncones[t];
    }
    if ((to && (!row || !col || !val)) || (tm && !b) || (tn && !c) || (tc && !cones))
        return bfail(nullptr, MFS_ERR_INVALID, "NULL array");
    for (int64_t i = 0; i < tm; ++i)
        if (!std::isfinite(b[i])) return bfail(nullptr, MFS_ERR_INVALID, "non-finite value in b");
    for (int64_t j = 0; j < tn; ++j)
        if (!std::isfinite(c[j])) return bfail(nullptr, MFS_ERR_INVALID, "non-finite value in c");

    mfs_batch* s = new (std::nothrow) mfs_batch();
    if (!s) return bfail(nullptr, MFS_ERR_OOM, "host allocation failed");
    auto bail = [&](mfs_status st) {
        g_batch_create_error = s->last_error;
        mfs_batch_destroy(s);
        return st;
    };
    s->set = set;
    s->count = (int)count;
    s->tune.threads = 256;
    s->tune.ctas_per_sm = 1;
    s->tune.check_every = set.check_every;
    // per instance: column order (rows ascending within a column) and row order, local indices.
    // Cones and offsets first (sequential, cheap), then the instances' orders in parallel, then
    // the concatenation.
    std::vector<int> hm(count), hn(count), ho(count), hns(count), cp, rp, ci, ri, sst, ssz;
    std::vector<long long> offn(count), offm(count), offo(count), offs(count);
    std::vector<int64_t> offz(count + 1, 0);
    std::vector<double> cv, rv;
    int64_t pn = 0, pm = 0, pc = 0;
    for (int64_t t = 0; t < count; ++t) {
        const int64_t nt = n[t];
        offn[t] = pn;
        offm[t] = pm;
        offs[t] = (long long)sst.size();
        offz[t + 1] = offz[t] + nnz[t];
        int64_t covered = 0;
        for (int64_t q = 0; q < ncones[t]; ++q) {
            const mfs_cone& cq = cones[pc + q];
            if (cq.size < 1 || (cq.kind != MFS_CONE_NONNEG && cq.kind != MFS_CONE_SOC)) {
                s->last_error = "bad cone in instance " + std::to_string(t);
                return bail(MFS_ERR_INVALID);
            }
            if (cq.kind == MFS_CONE_SOC) {
                sst.push_back((int)covered);
                ssz.push_back((int)cq.size);
            }
            covered += cq.size;
        }
        if (covered != nt) {
            s->last_error = "cone sizes do not sum to n in instance " + std::to_string(t);
            return bail(MFS_ERR_INVALID);
        }
        hns[t] = (int)(sst.size() - offs[t]);
        pc += ncones[t];
        hm[t] = (int)m[t];
        hn[t] = (int)nt;
        pn += nt;
        pm += m[t];
    }
    struct Orders {
        std::vector<int> cnt, ci, rc, ri;  // column pointers, rows (column order), row pointers, columns (row order)
        std::vector<double> cv, rv;
        int64_t bad = -1;                   // first bad entry, or -1
    };
    std::vector<Orders> ords(count);
    std::atomic<int64_t> next{0};
    const int nthr = mfs::host::threads_for(offz[count]);
    mfs::host::parallel_tasks(nthr, [&](int) {
        for (int64_t t = next++; t < count; t = next++) {
            Orders& R = ords[t];
            const int64_t mt = m[t], nt = n[t], kt = nnz[t], pz = offz[t];
            for (int64_t k = 0; k < kt && R.bad < 0; ++k) {
                const int64_t r = row[pz + k], q = col[pz + k];
                if (r < 0 || r >= mt || q < 0 || q >= nt || !std::isfinite(val[pz + k])) R.bad = k;
            }
            if (R.bad >= 0) continue;
            // sort the entries by (col, row) unless they already are; sum duplicates, drop zeros
            std::vector<int64_t> idx(kt);
            std::iota(idx.begin(), idx.end(), 0);
            bool sorted = true;
            for (int64_t k = 1; k < kt && sorted; ++k)
                sorted = col[pz + k - 1] < col[pz + k] || (col[pz + k - 1] == col[pz + k] && row[pz + k - 1] < row[pz + k]);
            if (!sorted)
                std::sort(idx.begin(), idx.end(), [&](int64_t p, int64_t q) {
                    return col[pz + p] != col[pz + q] ? col[pz + p] < col[pz + q] : row[pz + p] < row[pz + q];
                });
            std::vector<int> lc;
            R.ci.reserve(kt);
            R.cv.reserve(kt);
            lc.reserve(kt);
            for (int64_t k = 0; k < kt;) {
                const int64_t r = row[pz + idx[k]], q = col[pz + idx[k]];
                double a = 0.0;
                while (k < kt && row[pz + idx[k]] == r && col[pz + idx[k]] == q) a += val[pz + idx[k++]];
                if (a != 0.0) {
                    R.ci.push_back((int)r);
                    lc.push_back((int)q);
                    R.cv.push_back(a);
                }
            }
            const int ot = (int)R.cv.size();
            R.cnt.assign(nt + 1, 0);
            for (int k = 0; k < ot; ++k) R.cnt[lc[k] + 1]++;
            for (int64_t j = 0; j < nt; ++j) R.cnt[j + 1] += R.cnt[j];
            // row order (columns ascending within a row)
            R.rc.assign(mt + 1, 0);
            for (int k = 0; k < ot; ++k) R.rc[R.ci[k] + 1]++;
            for (int64_t i = 0; i < mt; ++i) R.rc[i + 1] += R.rc[i];
            std::vector<int> fill(R.rc.begin(), R.rc.begin() + mt);
            R.ri.resize(ot);
            R.rv.resize(ot);
            for (int k = 0; k < ot; ++k) {
                const int dst = fill[R.ci[k]]++;
                R.ri[dst] = lc[k];
                R.rv[dst] = R.cv[k];
            }
        }
    });
    for (int64_t t = 0; t < count; ++t)
        if (ords[t].bad >= 0) {
            s->last_error = "bad entry " + std::to_string(ords[t].bad) + " in instance " + std::to_string(t);
            return bail(MFS_ERR_INVALID);
        }
    int64_t po = 0;
    for (int64_t t = 0; t < count; ++t) {
        offo[t] = po;
        ho[t] = (int)ords[t].cv.size();
        po += ho[t];
    }
    cp.resize(tn + count);
    rp.resize(tm + count);
    ci.resize(po);
    ri.resize(po);
    cv.resize(po);
    rv.resize(po);
    mfs::host::parallel_ranges(count, nthr, [&](int64_t lo, int64_t hi, int) {
        for (int64_t t = lo; t < hi; ++t) {
            const Orders& R = ords[t];
            std::copy(R.cnt.begin(), R.cnt.end(), cp.begin() + offn[t] + t);
            std::copy(R.rc.begin(), R.rc.end(), rp.begin() + offm[t] + t);
            std::copy(R.ci.begin(), R.ci.end(), ci.begin() + offo[t]);
            std::copy(R.cv.begin(), R.cv.end(), cv.begin() + offo[t]);
            std::copy(R.ri.begin(), R.ri.end(), ri.begin() + offo[t]);
            std::copy(R.rv.begin(), R.rv.end(), rv.begin() + offo[t]);
        }
    });
    std::vector<Orders>().swap(ords);
    s->tot_n = pn;
    s->tot_m = pm;
    s->tot_o = po;
    s->tot_soc = (int64_t)sst.size();
    s->hm = hm;
    s->hn = hn;
    s->ho = ho;
    s->hoff_n = offn;
    s->hoff_m = offm;
    s->hoff_o = offo;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->max_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&s->max_smem_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    for (const void* f : {(const void*)k_batch<float, int, 0>, (const void*)k_batch<float, int, 1>,
                          (const void*)k_batch<float, int, 2>, (const void*)k_batch<double, int, 0>,
                          (const void*)k_batch<double, int, 1>, (const void*)k_batch<double, int, 2>,
                          (const void*)k_batch<float, uint16_t, 0>, (const void*)k_batch<float, uint16_t, 1>,
                          (const void*)k_batch<float, uint16_t, 2>, (const void*)k_batch<double, uint16_t, 0>,
                          (const void*)k_batch<double, uint16_t, 1>, (const void*)k_batch<double, uint16_t, 2>}) {
        cudaFuncAttributes fa;
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
        if (e == cudaSuccess) s->static_smem = std::max(s->static_smem, (int)fa.sharedSizeBytes);
    }
    if (e == cudaSuccess) {
        if (cuda_stream) {
            s->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = true;
        }
    }
    if (e != cudaSuccess) {
        s->last_error = std::string("CUDA set-up: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
    // largest instances first
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return ho[p] + hn[p] > ho[q] + hn[q]; });
#define BCHK(x)                             \
    do {                                    \
        mfs_status q_ = (x);                \
        if (q_ != MFS_OK) return bail(q_);  \
    } while (0)
    BCHK(bupload(s, &s->order, order.data(), order.size()));
    BCHK(bupload(s, &s->m, hm.data(), hm.size()));
    BCHK(bupload(s, &s->n, hn.data(), hn.size()));
    BCHK(bupload(s, &s->o, ho.data(), ho.size()));
    BCHK(bupload(s, &s->nsoc, hns.data(), hns.size()));
    BCHK(bupload(s, &s->off_n, offn.data(), offn.size()));
    BCHK(bupload(s, &s->off_m, offm.data(), offm.size()));
    BCHK(bupload(s, &s->off_o, offo.data(), offo.size()));
    BCHK(bupload(s, &s->off_soc, offs.data(), offs.size()));
    BCHK(bupload(s, &s->col_ptr, cp.data(), cp.size()));
    BCHK(bupload(s, &s->row_ptr, rp.data(), rp.size()));
    // local indices as 16 bits where every instance allows it (a quarter less to read per nonzero
    // and order, and more instances' matrices fit in shared memory), else 32
    s->idx16 = *std::max_element(hm.begin(), hm.end()) <= 65535 && *std::max_element(hn.begin(), hn.end()) <= 65535;
    if (s->idx16) {
        std::vector<uint16_t> c16(ci.begin(), ci.end()), r16(ri.begin(), ri.end());
        BCHK(bupload(s, &s->cidx16, c16.data(), c16.size()));
        BCHK(bupload(s, &s->ridx16, r16.data(), r16.size()));
    } else {
        BCHK(bupload(s, &s->cidx, ci.data(), ci.size()));
        BCHK(bupload(s, &s->ridx, ri.data(), ri.size()));
    }
    BCHK(bupload(s, &s->soc_start, sst.data(), sst.size()));
    BCHK(bupload(s, &s->soc_size, ssz.data(), ssz.size()));
    BCHK(bzeros(s, &s->queue, 1));
    BCHK(bzeros(s, &s->iters_done, count));
    BCHK(bzeros(s, &s->status, count));
    BCHK(bzeros(s, &s->resid, (size_t)count * NSTAT));
    if (set.precision == MFS_FP32_MIXED)
        BCHK(alloc_store<float>(s, s->f32, cv, rv, rp, b, c));
    else
        BCHK(alloc_store<double>(s, s->f64, cv, rv, rp, b, c));
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        s->last_error = std::string("set-up: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
#undef BCHK
    *out = s;
    return MFS_OK;
}

void mfs_batch_destroy(mfs_batch* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    if (s->graph) cudaGraphExecDestroy(s->graph);
    for (void* p : s->allocs) cudaFree(p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char* mfs_batch_last_error(const mfs_batch* s) {
    return s ? s->last_error.c_str() : g_batch_create_error.c_str();
}

mfs_status mfs_batch_set_tuning(mfs_batch* s, const mfs_batch_tuning* t) {
    if (!s || !t) return MFS_ERR_INVALID;
    if ((t->threads != 128 && t->threads != 256 && t->threads != 512) || t->ctas_per_sm < 1 || t->ctas_per_sm > 4 ||
        t->check_every < 1)
        return bfail(s, MFS_ERR_INVALID, "tuning: threads in {128,256,512}, ctas_per_sm in 1..4, check_every >= 1");
    s->tune = *t;
    s->set.check_every = t->check_every;
    if (s->graph) cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
    return MFS_OK;
}

mfs_status mfs_batch_get_tuning(const mfs_batch* s, mfs_batch_tuning* t) {
    if (!s || !t) return MFS_ERR_INVALID;
    *t = s->tune;
    return MFS_OK;
}

mfs_status mfs_batch_iterate(mfs_batch* s, int64_t k) {
    MFS_TRACE("mfs_batch_iterate");
    if (!s || k < 0 || k >= INT32_MAX) return MFS_ERR_INVALID;
    if (k == 0) return MFS_OK;
    BCUDA(s, cudaSetDevice(s->device));
    return s->set.precision == MFS_FP64 ? run_batch(s, s->f64, (int)k, 0.0) : run_batch(s, s->f32, (int)k, 0.0);
}

mfs_status mfs_batch_solve(mfs_batch* s, double tol, int64_t max_iter, int64_t* iters, int32_t* status) {
    MFS_TRACE("mfs_batch_solve");
    if (!s || !(tol > 0.0) || max_iter < 1 || max_iter >= INT32_MAX) return MFS_ERR_INVALID;
    BCUDA(s, cudaSetDevice(s->device));
    BCUDA(s, cudaMemsetAsync(s->iters_done, 0, sizeof(long long) * s->count, s->stream));
    BTRY(s->set.precision == MFS_FP64 ? run_batch(s, s->f64, (int)max_iter, tol)
                                      : run_batch(s, s->f32, (int)max_iter, tol));
    if (iters) {
        std::vector<long long> h(s->count);
        BCUDA(s, cudaMemcpy(h.data(), s->iters_done, sizeof(long long) * s->count, cudaMemcpyDeviceToHost));
        for (int t = 0; t < s->count; ++t) iters[t] = h[t];
    }
    if (status) {
        std::vector<int> h(s->count);
        BCUDA(s, cudaMemcpy(h.data(), s->status, sizeof(int) * s->count, cudaMemcpyDeviceToHost));
        for (int t = 0; t < s->count; ++t) status[t] = h[t] ? MFS_MAX_ITER : MFS_OK;
    }
    return MFS_OK;
}

mfs_status mfs_batch_residuals(mfs_batch* s, mfs_residuals_t* out) {
    if (!s || !out) return MFS_ERR_INVALID;
    BCUDA(s, cudaSetDevice(s->device));
    BTRY((s->set.precision == MFS_FP64 ? launch_batch<double, 1>(s, s->f64, 0, 0.0, s->stream)
                                       : launch_batch<float, 1>(s, s->f32, 0, 0.0, s->stream)));
    std::vector<double> h((size_t)s->count * NSTAT);
    std::vector<long long> it(s->count);
    BCUDA(s, cudaMemcpyAsync(h.data(), s->resid, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    BCUDA(s, cudaMemcpyAsync(it.data(), s->iters_done, it.size() * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
    BCUDA(s, cudaStreamSynchronize(s->stream));
    for (int t = 0; t < s->count; ++t) {
        double* d = reinterpret_cast<double*>(&out[t]);
        for (int q = 0; q < NSTAT; ++q) d[q] = h[(size_t)t * NSTAT + q];
        mfs::stop_measures(&out[t], s->set.osqp_rel);
        out[t].iter = it[t];
    }
    return MFS_OK;
}

mfs_status mfs_batch_get_solution(mfs_batch* s, int64_t t, double* x, double* lambda, double* z, double* delta) {
    if (!s || t < 0 || t >= s->count) return MFS_ERR_INVALID;
    BCUDA(s, cudaSetDevice(s->device));
    const int64_t n = s->hn[t], m = s->hm[t], gn = s->hoff_n[t], gm = s->hoff_m[t];
    double* tmp = nullptr;
    BCUDA(s, cudaMallocAsync((void**)&tmp, std::max<int64_t>(3 * n + m, 1) * sizeof(double), s->stream));
    auto get = [&](auto* src, int64_t off, int64_t cnt, double* dev, double* host) {
        if (!host || !cnt) return;
        k_to_double<<<(int)std::min<int64_t>((cnt + 255) / 256, 1024), 256, 0, s->stream>>>(dev, src + off, cnt);
        cudaMemcpyAsync(host, dev, cnt * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    };
    if (s->set.precision == MFS_FP64) {
        get(s->f64.x, gn, n, tmp, x);
        get(s->f64.lam, gm, m, tmp + n, lambda);
        get(s->f64.z, gn, n, tmp + n + m, z);
        get(s->f64.del, gn, n, tmp + 2 * n + m, delta);
    } else {
        get(s->f32.x, gn, n, tmp, x);
        get(s->f32.lam, gm, m, tmp + n, lambda);
        get(s->f32.z, gn, n, tmp + n + m, z);
        get(s->f32.del, gn, n, tmp + 2 * n + m, delta);
    }
    cudaFreeAsync(tmp, s->stream);
    BCUDA(s, cudaGetLastError());
    BCUDA(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_batch_index_bytes(const mfs_batch* s, int32_t* bytes) {
    if (!s || !bytes) return MFS_ERR_INVALID;
    *bytes = s->idx16 ? 2 : 4;
    return MFS_OK;
}

mfs_status mfs_batch_get_info(const mfs_batch* s, int64_t* count, int64_t* total_m, int64_t* total_n,
                              int64_t* total_nnz) {
    if (!s) return MFS_ERR_INVALID;
    if (count) *count = s->count;
    if (total_m) *total_m = s->tot_m;
    if (total_n) *total_n = s->tot_n;
    if (total_nnz) *total_nnz = s->tot_o;
    return MFS_OK;
}

mfs_status mfs_batch_tune(mfs_batch* s, int64_t iters, mfs_batch_tuning* chosen) {
    if (!s || iters < 1 || iters >= INT32_MAX) return MFS_ERR_INVALID;
    BCUDA(s, cudaSetDevice(s->device));
    // Time every candidate on the batch itself (the iterate advances) and keep the fastest.
    const mfs_batch_tuning keep = s->tune;
    mfs_batch_tuning best = keep;
    float best_ms = 1e30f;
    // events released on every return, including the early ones of a failed candidate
    struct Events {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ~Events() {
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
        }
    } ev;
    BCUDA(s, cudaEventCreate(&ev.e0));
    BCUDA(s, cudaEventCreate(&ev.e1));
    for (int threads : {128, 256, 512}) {
        for (int cps : {1, 2, 3, 4}) {
            mfs_batch_tuning t = keep;
            t.threads = threads;
            t.ctas_per_sm = cps;
            BTRY(mfs_batch_set_tuning(s, &t));
            BTRY(mfs_batch_iterate(s, 1));  // capture and warm
            cudaEventRecord(ev.e0, s->stream);
            BTRY(mfs_batch_iterate(s, iters));
            cudaEventRecord(ev.e1, s->stream);
            BCUDA(s, cudaEventSynchronize(ev.e1));
            float ms = 0;
            cudaEventElapsedTime(&ms, ev.e0, ev.e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    }
    // the residual-check interval: the smallest candidate whose in-launch FP64 checks cost at most
    // 5 % more than the sparsest one (no instance can meet the tolerance used here, so every
    // candidate runs all its iterations with all its checks); over at least two of the sparsest
    // candidate's intervals, so that every candidate's timing holds checks at its own spacing
    {
        const int cands[] = {10, 25, 50, 100, 200};
        const int64_t citers = std::max<int64_t>(iters, 2 * 200);
        float tc[5];
        for (int q = 0; q < 5; ++q) {
            mfs_batch_tuning t = best;
            t.check_every = cands[q];
            BTRY(mfs_batch_set_tuning(s, &t));
            BTRY(s->set.precision == MFS_FP64 ? run_batch(s, s->f64, (int)citers, 1e-300)
                                              : run_batch(s, s->f32, (int)citers, 1e-300));  // capture, warm
            cudaEventRecord(ev.e0, s->stream);
            BTRY(s->set.precision == MFS_FP64 ? run_batch(s, s->f64, (int)citers, 1e-300)
                                              : run_batch(s, s->f32, (int)citers, 1e-300));
            cudaEventRecord(ev.e1, s->stream);
            BCUDA(s, cudaEventSynchronize(ev.e1));
            cudaEventElapsedTime(&tc[q], ev.e0, ev.e1);
        }
        int pick = 4;
        for (int q = 3; q >= 0; --q)
            if (tc[q] <= 1.05f * tc[4]) pick = q;
        best.check_every = cands[pick];
    }
    BTRY(mfs_batch_set_tuning(s, &best));
    if (chosen) *chosen = best;
    return MFS_OK;
}

}  // extern "C"
