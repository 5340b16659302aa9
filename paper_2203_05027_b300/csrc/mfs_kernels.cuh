// mfs_kernels.cuh -- the per-iteration sweep and the FP64 residual reductions (sm_103a).
//
// Data layout (built on the host, see mfs_solver.cu): the nonzeros of A are kept twice, in
// column order (CSC: col_ptr plus padded row-index/value arrays) and in row order (CSR: row_ptr
// plus padded column-index/value arrays). Columns are grouped into chunks of at most WT = 256
// nonzeros and WC columns; a chunk never splits a Lorentz cone small enough to fit one, and a
// single column longer than WT is a "long" chunk of its own. Rows are chunked the same way. Each
// chunk starts at a multiple of PAD = 8 elements of the padded arrays, so one warp loads a whole
// chunk with one 256-bit load per lane and array (lane l holds local nonzeros 8l .. 8l+7).
//
// One warp owns one chunk: it gathers the other side's vector at its nonzeros' indices, reduces
// the products per column (warp-level segmented scan, no block barriers) and runs the column
// epilogue. Long chunks go to a CTA each.
//
// One iteration of the reduced form of Algorithm 1 (state x, z, delta, lambda and
// v = F_U (b - A x_prev) - lambda/mu) is
//   column sweep:  x_j <- (d_j x_j + sum_{k in col j} a_k v_{i_k} + z_j + (delta_j - c_j)/mu)/(1+d_j)
//                  z   <- proj_K(x - delta/mu) (eq. proj), delta <- delta + mu (z - x)
//   row sweep:     rho_i = (b_i - sum_{k in row i} a_k x_{j_k}) / (1 + sum_{k in row i} a_k^2)
//                  lambda_i <- lambda_i - mu rho_i,   v_i <- rho_i - lambda_i/mu
// (x-step eq. vvt with F_V = 1/(1+d); y-step with the matrix inversion lemma and F_U; the dual
// updates of Algorithm 1; gamma = -U^T lambda and y = V^T x + U^T rho are implied.)
#pragma once

#include <type_traits>

#include "mfs_device.cuh"
#include "mfs_measures.h"

// Minimum resident CTAs per SM requested for the FP32 sweep kernels (8 x 256 threads: 32 registers,
// more warps to keep gathers in flight). The FP64 sweeps, ALU-bound, keep their full register budget.
#ifndef MFS_SWEEP_MINB
#define MFS_SWEEP_MINB 8
#endif

namespace mfs {

template <typename T>
struct SweepArgs {
    // column order
    const int* __restrict__ col_ptr;  // n+1 offsets into the unpadded column order
    const int* __restrict__ cidx;     // padded row indices
    const T* __restrict__ cval;       // padded values
    const int4* __restrict__ cdesc;   // per column chunk: {first column, one past last, padded offset, nnz}
    const uint32_t* __restrict__ cheads;  // per column chunk: 8 words, bit e set if a column starts at local nonzero e
    const int* __restrict__ clong;    // indices of the long column chunks
    const int* __restrict__ cq_lo;    // per column chunk: first Lorentz cone intersecting it
    const int* __restrict__ cq_hi;    // one past the last such cone
    // row order
    const int* __restrict__ row_ptr;
    const int* __restrict__ ridx;
    const T* __restrict__ rval;
    const int4* __restrict__ rdesc;
    const uint32_t* __restrict__ rheads;
    const int* __restrict__ rlong;
    // Lorentz cones, in coordinate order
    const int* __restrict__ soc_start;
    const int* __restrict__ soc_size;
    const unsigned char* __restrict__ soc_big;  // 1: too large to fuse, handled by the big-cone kernel
    const int* __restrict__ big_list;           // indices of the big cones
    const unsigned char* __restrict__ ctag;     // per column: 0 orthant, 1 small Lorentz cone, 2 big cone
    // data and iterate
    const T* __restrict__ b;
    const T* __restrict__ c;
    T* x;
    T* z;
    T* del;
    T* lam;
    T* v;
    T mu;
    int ntc, ntr;      // column / row chunks
    int nlc, nlr;      // long column / row chunks
    int m, n;          // bounds of the checked build (gathered indices)
    long long cpad, rpad;  // lengths of the padded column / row nonzero arrays
};

template <typename T>
__device__ __forceinline__ T ldro(const T* p) {
    return __ldg(p);
}

// w[i] through the read-only path; in the checked build i is checked against lim first.
template <typename T>
__device__ __forceinline__ T gat(const T* __restrict__ w, int i, int lim, int site) {
    return MFS_INB(i, lim, site) ? __ldg(w + i) : T(0);
}

// Segment sums of one chunk held by one warp. heads: the chunk's 8-word start bitmap (bit e set
// if a non-empty segment begins at local nonzero e). prod(index, value, out[NV]) gives the
// per-nonzero terms. On return s_end[eslot(e)*NV + t] holds the sums of the segment whose last
// nonzero is local item e.
template <typename T, typename A, int NV, typename Prod>
__device__ __forceinline__ void warp_chunk_sums(const int* __restrict__ gidx, const T* __restrict__ gval, int koff,
                                                int nnz, const uint32_t* __restrict__ heads, A* s_end, Prod prod,
                                                long long pad) {
    const int lane = threadIdx.x & 31;
    const int e0 = lane * IPT;
    A p[IPT][NV];
    if (e0 < nnz && MFS_INB((long long)koff + e0 + IPT - 1, pad, BS_ENTRIES)) {
        int id[IPT];
        T vl[IPT];
        ld256(gidx + koff + e0, id);
        ld256(gval + koff + e0, vl);
#pragma unroll
        for (int q = 0; q < IPT; ++q) {
            if (e0 + q < nnz) {
                prod(id[q], vl[q], p[q]);
            } else {
#pragma unroll
                for (int t = 0; t < NV; ++t) p[q][t] = A(0);
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < IPT; ++q)
#pragma unroll
            for (int t = 0; t < NV; ++t) p[q][t] = A(0);
    }
    const int wi = lane >> 2;
    const uint64_t hw = (uint64_t)__ldg(heads + wi) | ((uint64_t)(wi < 7 ? __ldg(heads + wi + 1) : 0u) << 32);
    const uint32_t hb = (uint32_t)(hw >> ((lane & 3) * 8)) & 0x1FFu;  // items e0 .. e0+8
    Sums<A, NV> agg;
#pragma unroll
    for (int t = 0; t < NV; ++t) agg.v[t] = A(0);
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        if ((hb >> q) & 1u) {
#pragma unroll
            for (int t = 0; t < NV; ++t) agg.v[t] = p[q][t];
        } else {
#pragma unroll
            for (int t = 0; t < NV; ++t) agg.v[t] = agg.v[t] + p[q][t];
        }
    }
    Sums<A, NV> acc = warp_seg_carry<A, NV>((hb & 0xFFu) != 0u, agg);
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        const int e = e0 + q;
        if (e < nnz) {
            if ((hb >> q) & 1u) {
#pragma unroll
                for (int t = 0; t < NV; ++t) acc.v[t] = p[q][t];
            } else {
#pragma unroll
                for (int t = 0; t < NV; ++t) acc.v[t] = acc.v[t] + p[q][t];
            }
            if (e == nnz - 1 || ((hb >> (q + 1)) & 1u)) {
#pragma unroll
                for (int t = 0; t < NV; ++t) s_end[eslot(e) * NV + t] = acc.v[t];
            }
        }
    }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ T col_x_update(T d, T xprev, T atv, T zj, T dj, T cj, T mu) {
    return (d * xprev + atv + zj + (dj - cj) / mu) / (T(1) + d);
}

// Lorentz-cone projection of coordinate t of w (eq. proj), given w_1 and alpha = ||w_{2..}||.
template <typename T>
__device__ __forceinline__ T lorentz_coord(T w, int t, T w1, T alpha) {
    if (alpha <= -w1) return T(0);
    if (alpha <= w1) return w;
    return (t == 0) ? w / T(2) + alpha / T(2) : w / T(2) + w1 * w / (T(2) * alpha);
}

// Cone membership of column j: 0 orthant, 1 small Lorentz cone (fused), 2 Lorentz cone handled by
// the big-cone kernels (a byte per column, tabulated at set-up).
template <typename T>
__device__ __forceinline__ int cone_tag(const SweepArgs<T>& a, int j) {
    return __ldg(a.ctag + j);
}

// The small Lorentz cones of column chunk ch, in order: body(c0, size) for each (c0 its first column
// relative to lo), called by the whole warp. Their descriptors are loaded 32 at a time, one per
// lane, and handed round by shuffles, so that no cone waits for its own loads.
template <typename T, typename Body>
__device__ __forceinline__ void for_small_cones(const SweepArgs<T>& a, int ch, int lo, Body body) {
    const int lane = threadIdx.x & 31;
    const int qlo = a.cq_lo[ch], qhi = a.cq_hi[ch];
    for (int q0 = qlo; q0 < qhi; q0 += 32) {
        const int q = q0 + lane;
        int st = 0, sz = 0, big = 1;
        if (q < qhi) {
            st = a.soc_start[q];
            sz = a.soc_size[q];
            big = a.soc_big[q];
        }
        const int cnt = min(32, qhi - q0);
        for (int u = 0; u < cnt; ++u) {
            if (__shfl_sync(FULL, big, u)) continue;
            body(__shfl_sync(FULL, st, u) - lo, __shfl_sync(FULL, sz, u));
        }
    }
}

// x-, z- and delta-updates of one orthant column.
template <typename T>
__device__ __forceinline__ void orthant_update(T* x, T* z, T* del, int j, T xn, T dj, T mu) {
    x[j] = xn;
    const T w = xn - dj / mu;
    const T zn = w > T(0) ? w : T(0);
    z[j] = zn;
    del[j] = dj + mu * (zn - xn);
}

// ------------------------------------------------------------------------------------ column sweep
template <typename T, bool SOC>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? MFS_SWEEP_MINB : 1) k_col_sweep(const SweepArgs<T> a) {
    __shared__ T s_end[NWARP][ESLOTS];
    __shared__ T s_cone[SOC ? NWARP : 1][3][WC];  // x, w = x - delta/mu, delta of small-cone columns
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * NWARP + warp;
    if (ch >= a.ntc) return;
    const int4 dsc = a.cdesc[ch];
    const int lo = dsc.x, nseg = dsc.y - dsc.x, koff = dsc.z, nnz = dsc.w;
    if (nnz > WT) return;  // long chunk: k_col_long
    const T mu = a.mu;
    int cs[CPL], ce[CPL];
    T px[CPL], pz[CPL], pd[CPL], pc[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int jl = lane + 32 * k;
        cs[k] = ce[k] = 0;
        px[k] = pz[k] = pd[k] = pc[k] = T(0);
        if (jl < nseg) {
            const int j = lo + jl;
            cs[k] = a.col_ptr[j];
            ce[k] = a.col_ptr[j + 1];
            px[k] = a.x[j];
            pz[k] = a.z[j];
            pd[k] = a.del[j];
            pc[k] = a.c[j];
        }
    }
    const int kb = __shfl_sync(FULL, cs[0], 0);
    const T* __restrict__ v = a.v;
    const int m = a.m;
    auto prod = [v, m](int i, T val, T (&p)[1]) { p[0] = val * gat(v, i, m, BS_GATHER_V); };
    warp_chunk_sums<T, T, 1>(a.cidx, a.cval, koff, nnz, a.cheads + (size_t)ch * 8, s_end[warp], prod, a.cpad);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int jl = lane + 32 * k;
        if (jl < nseg) {
            const T atv = (ce[k] > cs[k]) ? s_end[warp][eslot(ce[k] - 1 - kb)] : T(0);
            const T xn = col_x_update(T(ce[k] - cs[k]), px[k], atv, pz[k], pd[k], pc[k], mu);
            const int j = lo + jl;
            const int tag = SOC ? cone_tag(a, j) : 0;
            if (tag == 0) {
                orthant_update(a.x, a.z, a.del, j, xn, pd[k], mu);
            } else {
                a.x[j] = xn;
                if (tag == 1) {
                    s_cone[SOC ? warp : 0][0][jl] = xn;
                    s_cone[SOC ? warp : 0][1][jl] = xn - pd[k] / mu;
                    s_cone[SOC ? warp : 0][2][jl] = pd[k];
                }
            }
        }
    }
    if (SOC) {
        __syncwarp();
        // the small cones of the chunk one after another, each by the whole warp: ||w_tail||^2 by a
        // butterfly sum, then the z-step (eq. proj) and delta-update of one coordinate per lane
        const T* cx = s_cone[warp][0];
        const T* cw = s_cone[warp][1];
        const T* cd = s_cone[warp][2];
        for_small_cones(a, ch, lo, [&](int c0, int sz) {
            T ss = T(0);
            for (int t = 1 + lane; t < sz; t += 32) ss += cw[c0 + t] * cw[c0 + t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(FULL, ss, o);
            const T alpha = sqrt(ss), w1 = cw[c0];
            for (int t = lane; t < sz; t += 32) {
                const T zt = lorentz_coord(cw[c0 + t], t, w1, alpha);
                a.z[lo + c0 + t] = zt;
                a.del[lo + c0 + t] = cd[c0 + t] + mu * (zt - cx[c0 + t]);
            }
        });
    }
}

// A column longer than one chunk: one CTA reduces it and runs its epilogue.
template <typename T, bool SOC>
__global__ void __launch_bounds__(NT) k_col_long(const SweepArgs<T> a) {
    __shared__ T sh[NWARP];
    const int ch = a.clong[blockIdx.x];
    const int4 dsc = a.cdesc[ch];
    const int j = dsc.x, koff = dsc.z, nnz = dsc.w;
    Sums<T, 1> s;
    s.v[0] = T(0);
    for (int e = threadIdx.x; e < nnz; e += NT)
        if (MFS_INB((long long)koff + e, a.cpad, BS_ENTRIES))
            s.v[0] += a.cval[koff + e] * gat(a.v, a.cidx[koff + e], a.m, BS_GATHER_V);
    s = block_sum<T, 1>(s, sh);
    if (threadIdx.x == 0) {
        const T mu = a.mu, dj = a.del[j];
        const T xn = col_x_update(T(nnz), a.x[j], s.v[0], a.z[j], dj, a.c[j], mu);
        if (SOC && cone_tag(a, j) != 0)  // then part of a big cone
            a.x[j] = xn;
        else
            orthant_update(a.x, a.z, a.del, j, xn, dj, mu);
    }
}

// z-step and delta-update of a Lorentz cone too large to fuse into the column sweep (one CTA per
// cone); x already holds the new x.
template <typename T>
__global__ void __launch_bounds__(NT) k_bigcone_sweep(const SweepArgs<T> a) {
    __shared__ T sh[NWARP];
    __shared__ T s_alpha;
    const int q = a.big_list[blockIdx.x];
    const int st = a.soc_start[q], sz = a.soc_size[q];
    const T mu = a.mu;
    Sums<T, 1> ss;
    ss.v[0] = T(0);
    for (int t = 1 + threadIdx.x; t < sz; t += NT) {
        const T w = a.x[st + t] - a.del[st + t] / mu;
        ss.v[0] += w * w;
    }
    ss = block_sum<T, 1>(ss, sh);
    if (threadIdx.x == 0) s_alpha = sqrt(ss.v[0]);
    __syncthreads();
    const T alpha = s_alpha;
    const T w1 = a.x[st] - a.del[st] / mu;
    for (int t = threadIdx.x; t < sz; t += NT) {
        const T xt = a.x[st + t], dt = a.del[st + t];
        const T zt = lorentz_coord(xt - dt / mu, t, w1, alpha);
        a.z[st + t] = zt;
        a.del[st + t] = dt + mu * (zt - xt);
    }
}

// ------------------------------------------------------------------------------------ row sweep
// MODE 0: iteration (lambda and v updated). MODE 1: v from x and the current lambda (warm start,
// change of mu).
template <typename T, int MODE>
__device__ __forceinline__ void row_update(const SweepArgs<T>& a, int i, T ax, T r, T bi, T li) {
    const T mu = a.mu;
    const T rho = (bi - ax) / (T(1) + r);
    if (MODE == 0) {
        const T ln = li - mu * rho;
        a.lam[i] = ln;
        a.v[i] = rho - ln / mu;
    } else {
        a.v[i] = rho - li / mu;
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? MFS_SWEEP_MINB : 1) k_row_sweep(const SweepArgs<T> a) {
    __shared__ T s_end[NWARP][2 * ESLOTS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ch = blockIdx.x * NWARP + warp;
    if (ch >= a.ntr) return;
    const int4 dsc = a.rdesc[ch];
    const int lo = dsc.x, nseg = dsc.y - dsc.x, koff = dsc.z, nnz = dsc.w;
    if (nnz > WT) return;  // long chunk: k_row_long
    int cs[CPL], ce[CPL];
    T pb[CPL], pl[CPL];
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int il = lane + 32 * k;
        cs[k] = ce[k] = 0;
        pb[k] = pl[k] = T(0);
        if (il < nseg) {
            const int i = lo + il;
            cs[k] = a.row_ptr[i];
            ce[k] = a.row_ptr[i + 1];
            pb[k] = a.b[i];
            pl[k] = a.lam[i];
        }
    }
    const int kb = __shfl_sync(FULL, cs[0], 0);
    const T* __restrict__ x = a.x;
    const int n = a.n;
    auto prod = [x, n](int j, T val, T (&p)[2]) {
        p[0] = val * gat(x, j, n, BS_GATHER_X);
        p[1] = val * val;
    };
    warp_chunk_sums<T, T, 2>(a.ridx, a.rval, koff, nnz, a.rheads + (size_t)ch * 8, s_end[warp], prod, a.rpad);
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int il = lane + 32 * k;
        if (il < nseg) {
            const bool ne = ce[k] > cs[k];
            const int e = eslot(ce[k] - 1 - kb);
            row_update<T, MODE>(a, lo + il, ne ? s_end[warp][2 * e] : T(0), ne ? s_end[warp][2 * e + 1] : T(0), pb[k],
                                pl[k]);
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(NT) k_row_long(const SweepArgs<T> a) {
    __shared__ T sh[2 * NWARP];
    const int ch = a.rlong[blockIdx.x];
    const int4 dsc = a.rdesc[ch];
    const int i = dsc.x, koff = dsc.z, nnz = dsc.w;
    Sums<T, 2> s;
    s.v[0] = s.v[1] = T(0);
    for (int e = threadIdx.x; e < nnz; e += NT) {
        if (!MFS_INB((long long)koff + e, a.rpad, BS_ENTRIES)) continue;
        const T val = a.rval[koff + e];
        s.v[0] += val * gat(a.x, a.ridx[koff + e], a.n, BS_GATHER_X);
        s.v[1] += val * val;
    }
    s = block_sum<T, 2>(s, sh);
    if (threadIdx.x == 0) row_update<T, MODE>(a, i, s.v[0], s.v[1], a.b[i], a.lam[i]);
}

// ------------------------------------------------------------------------------------ residuals
// Per-nonzero products and per-segment sums of the residual kernels: exact FP32 products summed
// as float pairs when the data are FP32 (then converted to FP64), plain FP64 when they are FP64.
template <typename T>
struct AccOf {
    using type = DF;
};
template <>
struct AccOf<double> {
    using type = double;
};

__device__ __forceinline__ DF acc_prod(float a, float b) {
    return df_prod(a, b);
}
__device__ __forceinline__ double acc_prod(double a, double b) {
    return a * b;
}

// Sum of a_k * w[idx_k] over one long segment by one warp (lane-strided, fixed order).
template <typename T>
__device__ __forceinline__ double warp_long_dot(const int* __restrict__ gidx, const T* __restrict__ gval, int koff,
                                                int nnz, const T* __restrict__ w, long long pad, int lim, int site) {
    using A = typename AccOf<T>::type;
    const int lane = threadIdx.x & 31;
    A acc = A(0);
    for (int e = lane; e < nnz; e += 32)
        if (MFS_INB((long long)koff + e, pad, BS_ENTRIES))
            acc = acc + acc_prod(gval[koff + e], gat(w, gidx[koff + e], lim, site));
    double d = to_double(acc);
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) d += __shfl_xor_sync(FULL, d, k);
    return d;
}

// Row-side fields (sums of squares and maxima of |.|), column-side fields and big-cone fields;
// each residual CTA writes one value per field, field-major: part[f * grid + cta].
enum : int { R_RES2 = 0, R_RESMAX, R_AXMAX, R_B2, R_BMAX, R_BLAM, NFR };
enum : int { C_S2 = 0, C_SMAX, C_ATLMAX, C_C2, C_CMAX, C_CX, C_X2, C_SDIST2, C_XDIST2, C_XMAX, C_SDMAX, C_XDMAX, NFC };
enum : int { B_SDIST2 = 0, B_XDIST2, B_SDMAX, B_XDMAX, NFB };

__host__ __device__ constexpr bool row_field_is_max(int f) {
    return f == R_RESMAX || f == R_AXMAX || f == R_BMAX;
}
__host__ __device__ constexpr bool col_field_is_max(int f) {
    return f == C_SMAX || f == C_ATLMAX || f == C_CMAX || f == C_XMAX || f == C_SDMAX || f == C_XDMAX;
}
__host__ __device__ constexpr bool big_field_is_max(int f) {
    return f == B_SDMAX || f == B_XDMAX;
}

// Squared distance of w to one Lorentz cone, given w_1 and alpha = ||w_{2..}||
// (w - P(w) is 0, w, or has norm^2 (alpha - w_1)^2 / 2 in the three cases of eq. proj).
__device__ __forceinline__ double lorentz_dist2(double w1, double alpha, double wnorm2) {
    if (alpha <= -w1) return wnorm2;
    if (alpha <= w1) return 0.0;
    const double g = alpha - w1;
    return 0.5 * g * g;
}

// Fold the lanes' NFIELD accumulators into one value per field for the CTA (fixed order).
template <int NFIELD, bool ROW>
__device__ __forceinline__ bool field_max(int k) {
    return ROW ? row_field_is_max(k) : col_field_is_max(k);
}

template <int NFIELD, bool ROW>
__device__ __forceinline__ void cta_fields_out(double (&f)[NFIELD], double (*sh)[NFIELD], double* part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NFIELD; ++k) {
        double v = f[k];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const double o = __shfl_down_sync(FULL, v, d);
            v = field_max<NFIELD, ROW>(k) ? fmax(v, o) : v + o;
        }
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NFIELD) {
        const int k = threadIdx.x;
        double acc = 0.0;
        for (int w = 0; w < NWARP; ++w) acc = field_max<NFIELD, ROW>(k) ? fmax(acc, sh[w][k]) : acc + sh[w][k];
        part[(size_t)k * gridDim.x + blockIdx.x] = acc;
    }
}

// Per-lane residual fields of the FP32 iterate as double-float pairs (about 48 significant bits):
// B300 runs FP64 at 1/64 of its FP32 rate, and FP64 arithmetic per column or row was the larger
// part of the residual kernels' time. Each lane folds its pairs into FP64 once, before the FP64
// reductions over the CTA and the grid. Maxima compare normalised pairs (hi first, then lo).
template <typename A>
__device__ __forceinline__ A acc_from(double d);
template <>
__device__ __forceinline__ DF acc_from<DF>(double d) {
    return df_from(d);
}
template <>
__device__ __forceinline__ double acc_from<double>(double d) {
    return d;
}

// Fold a lane's pair fields into its FP64 fields (sums added, maxima taken).
template <int NFIELD, bool ROW>
__device__ __forceinline__ void fold_df_fields(double (&f)[NFIELD], const DF (&F)[NFIELD]) {
#pragma unroll
    for (int k = 0; k < NFIELD; ++k) {
        const double v = to_double(F[k]);
        f[k] = field_max<NFIELD, ROW>(k) ? fmax(f[k], v) : f[k] + v;
    }
}

struct ResidArgs {
    double* part_row;  // NFR x (row-residual grid)
    double* part_col;  // NFC x (column-residual grid)
    double* part_big;  // NFB x (big cones)
    double* s_buf;     // n: c + A^T lambda (FP64), written for big-cone columns (all if write_all_s)
    double* r_buf;     // m: A x - b (FP64), written if write_all_s
    int write_all_s;
};

// Row-side residual fields: ||Ax - b||, max|Ax - b|, max|Ax|, ||b||, max|b|, b^T lambda, reduced in
// FP64 (per lane as double-float pairs for the FP32 iterate).
// Persistent warps walk the row chunks.
template <typename T>
__global__ void __launch_bounds__(NT) k_row_resid(const SweepArgs<T> a, const ResidArgs r) {
    using A = typename AccOf<T>::type;
    __shared__ A s_end[NWARP][ESLOTS];
    __shared__ double s_red[NWARP][NFR];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool F32 = std::is_same<T, float>::value;
    double f[NFR];
    DF F[F32 ? NFR : 1];
#pragma unroll
    for (int k = 0; k < NFR; ++k) f[k] = 0.0;
#pragma unroll
    for (int k = 0; k < (F32 ? NFR : 1); ++k) F[k] = DF(0);
    const T* __restrict__ x = a.x;
    const int n = a.n;
    auto prod = [x, n](int j, T val, A (&p)[1]) { p[0] = acc_prod(val, gat(x, j, n, BS_GATHER_XR)); };
    for (int ch = blockIdx.x * NWARP + warp; ch < a.ntr; ch += gridDim.x * NWARP) {
        const int4 dsc = a.rdesc[ch];
        const int lo = dsc.x, nseg = dsc.y - dsc.x, koff = dsc.z, nnz = dsc.w;
        A ax[CPL];
        int rows[CPL];
        if (nnz > WT) {  // one long row: the warp sums it
            ax[0] = acc_from<A>(warp_long_dot(a.ridx, a.rval, koff, nnz, x, a.rpad, a.n, BS_GATHER_XR));
            rows[0] = (lane == 0) ? lo : -1;
#pragma unroll
            for (int k = 1; k < CPL; ++k) rows[k] = -1;
        } else {
            int cs[CPL], ce[CPL];
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const int il = lane + 32 * k;
                cs[k] = ce[k] = 0;
                if (il < nseg) {
                    cs[k] = a.row_ptr[lo + il];
                    ce[k] = a.row_ptr[lo + il + 1];
                }
            }
            const int kb = __shfl_sync(FULL, cs[0], 0);
            warp_chunk_sums<T, A, 1>(a.ridx, a.rval, koff, nnz, a.rheads + (size_t)ch * 8, s_end[warp], prod, a.rpad);
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const int il = lane + 32 * k;
                rows[k] = il < nseg ? lo + il : -1;
                ax[k] = (il < nseg && ce[k] > cs[k]) ? s_end[warp][eslot(ce[k] - 1 - kb)] : A(0);
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            if (rows[k] < 0) continue;
            if constexpr (F32) {
                const float bi = a.b[rows[k]];
                const DF res = ax[k] + DF(-bi, 0.f);
                if (r.write_all_s) r.r_buf[rows[k]] = to_double(res);
                F[R_RES2] = F[R_RES2] + df_sq(res);
                F[R_RESMAX] = df_max(F[R_RESMAX], df_abs(res));
                F[R_AXMAX] = df_max(F[R_AXMAX], df_abs(ax[k]));
                F[R_B2] = F[R_B2] + df_prod(bi, bi);
                F[R_BMAX] = df_max(F[R_BMAX], DF(fabsf(bi), 0.f));
                F[R_BLAM] = F[R_BLAM] + df_prod(bi, a.lam[rows[k]]);
            } else {
                const double axk = to_double(ax[k]);
                const double bi = double(a.b[rows[k]]), res = axk - bi;
                if (r.write_all_s) r.r_buf[rows[k]] = res;
                f[R_RES2] += res * res;
                f[R_RESMAX] = fmax(f[R_RESMAX], fabs(res));
                f[R_AXMAX] = fmax(f[R_AXMAX], fabs(axk));
                f[R_B2] += bi * bi;
                f[R_BMAX] = fmax(f[R_BMAX], fabs(bi));
                f[R_BLAM] += bi * double(a.lam[rows[k]]);
            }
        }
    }
    if constexpr (F32) fold_df_fields<NFR, true>(f, F);
    cta_fields_out<NFR, true>(f, s_red, r.part_row);
}

// Column-side residual fields (reduced like the row side): with s = c + A^T lambda, ||s||, max|s|, max|A^T lambda|,
// ||c||, max|c|, c^T x, ||x||, dist(s, K)^2 and dist(x, K)^2 (small cones fused; big cones get s
// in s_buf for k_bigcone_resid). Persistent warps walk the column chunks.
template <typename T, bool SOC>
__global__ void __launch_bounds__(NT) k_col_resid(const SweepArgs<T> a, const ResidArgs r) {
    using A = typename AccOf<T>::type;
    __shared__ A s_end[NWARP][ESLOTS];
    __shared__ double s_red[NWARP][NFC];
    __shared__ double s_cone[SOC ? NWARP : 1][2][WC];  // s and x of small-cone columns
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool F32 = std::is_same<T, float>::value;
    double f[NFC];  // FP64 path; for the FP32 iterate the Lorentz-cone terms only
    DF F[F32 ? NFC : 1];
#pragma unroll
    for (int k = 0; k < NFC; ++k) f[k] = 0.0;
#pragma unroll
    for (int k = 0; k < (F32 ? NFC : 1); ++k) F[k] = DF(0);
    const T* __restrict__ lam = a.lam;
    const int m = a.m;
    auto prod = [lam, m](int i, T val, A (&p)[1]) { p[0] = acc_prod(val, gat(lam, i, m, BS_GATHER_L)); };
    for (int ch = blockIdx.x * NWARP + warp; ch < a.ntc; ch += gridDim.x * NWARP) {
        const int4 dsc = a.cdesc[ch];
        const int lo = dsc.x, nseg = dsc.y - dsc.x, koff = dsc.z, nnz = dsc.w;
        A atl[CPL];
        int cols[CPL];
        if (nnz > WT) {  // one long column: the warp sums it
            atl[0] = acc_from<A>(warp_long_dot(a.cidx, a.cval, koff, nnz, lam, a.cpad, a.m, BS_GATHER_L));
            cols[0] = (lane == 0) ? 0 : -1;
#pragma unroll
            for (int k = 1; k < CPL; ++k) cols[k] = -1;
        } else {
            int cs[CPL], ce[CPL];
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const int jl = lane + 32 * k;
                cs[k] = ce[k] = 0;
                if (jl < nseg) {
                    cs[k] = a.col_ptr[lo + jl];
                    ce[k] = a.col_ptr[lo + jl + 1];
                }
            }
            const int kb = __shfl_sync(FULL, cs[0], 0);
            warp_chunk_sums<T, A, 1>(a.cidx, a.cval, koff, nnz, a.cheads + (size_t)ch * 8, s_end[warp], prod, a.cpad);
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const int jl = lane + 32 * k;
                cols[k] = jl < nseg ? jl : -1;
                atl[k] = (jl < nseg && ce[k] > cs[k]) ? s_end[warp][eslot(ce[k] - 1 - kb)] : A(0);
            }
            __syncwarp();
        }
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int jl = cols[k];
            if (jl < 0) continue;
            const int j = lo + jl;
            const int tag = SOC ? cone_tag(a, j) : 0;
            double s;  // written for the cone kernels only (FP32 iterate)
            if constexpr (F32) {
                const float cj = a.c[j], xj = a.x[j];
                const DF sd = DF(cj, 0.f) + atl[k];
                F[C_S2] = F[C_S2] + df_sq(sd);
                F[C_SMAX] = df_max(F[C_SMAX], df_abs(sd));
                F[C_ATLMAX] = df_max(F[C_ATLMAX], df_abs(atl[k]));
                F[C_C2] = F[C_C2] + df_prod(cj, cj);
                F[C_CMAX] = df_max(F[C_CMAX], DF(fabsf(cj), 0.f));
                F[C_CX] = F[C_CX] + df_prod(cj, xj);
                F[C_X2] = F[C_X2] + df_prod(xj, xj);
                F[C_XMAX] = df_max(F[C_XMAX], DF(fabsf(xj), 0.f));
                if (tag == 0) {
                    const DF sn = sd.hi < 0.f ? sd : DF(0);
                    const float xn = xj < 0.f ? xj : 0.f;
                    F[C_SDIST2] = F[C_SDIST2] + df_sq(sn);
                    F[C_XDIST2] = F[C_XDIST2] + df_prod(xn, xn);
                    F[C_SDMAX] = df_max(F[C_SDMAX], df_neg(sn));
                    F[C_XDMAX] = df_max(F[C_XDMAX], DF(-xn, 0.f));
                }
                s = (tag != 0 || r.write_all_s) ? to_double(sd) : 0.0;
                if (tag == 1) {
                    s_cone[SOC ? warp : 0][0][jl] = s;
                    s_cone[SOC ? warp : 0][1][jl] = double(xj);
                }
            } else {
                const double cj = double(a.c[j]), xj = double(a.x[j]);
                s = cj + atl[k];
                f[C_S2] += s * s;
                f[C_SMAX] = fmax(f[C_SMAX], fabs(s));
                f[C_ATLMAX] = fmax(f[C_ATLMAX], fabs(atl[k]));
                f[C_C2] += cj * cj;
                f[C_CMAX] = fmax(f[C_CMAX], fabs(cj));
                f[C_CX] += cj * xj;
                f[C_X2] += xj * xj;
                f[C_XMAX] = fmax(f[C_XMAX], fabs(xj));
                if (tag == 0) {
                    const double sn = s < 0.0 ? s : 0.0, xn = xj < 0.0 ? xj : 0.0;
                    f[C_SDIST2] += sn * sn;
                    f[C_XDIST2] += xn * xn;
                    f[C_SDMAX] = fmax(f[C_SDMAX], -sn);
                    f[C_XDMAX] = fmax(f[C_XDMAX], -xn);
                } else if (tag == 1) {
                    s_cone[SOC ? warp : 0][0][jl] = s;
                    s_cone[SOC ? warp : 0][1][jl] = xj;
                }
            }
            if (tag == 2 || r.write_all_s) r.s_buf[j] = s;
        }
        if (SOC && nnz <= WT) {
            __syncwarp();
            const double* cs_ = s_cone[warp][0];
            const double* cx_ = s_cone[warp][1];
            for_small_cones(a, ch, lo, [&](int c0, int sz) {  // each small cone by the whole warp
                double ss = 0.0, xx = 0.0;
                for (int t = 1 + lane; t < sz; t += 32) {
                    ss += cs_[c0 + t] * cs_[c0 + t];
                    xx += cx_[c0 + t] * cx_[c0 + t];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ss += __shfl_xor_sync(FULL, ss, o);
                    xx += __shfl_xor_sync(FULL, xx, o);
                }
                if (lane == 0) {
                    const double s1 = cs_[c0], x1 = cx_[c0];
                    const double as = sqrt(ss), ax = sqrt(xx);
                    f[C_SDIST2] += lorentz_dist2(s1, as, ss + s1 * s1);
                    f[C_XDIST2] += lorentz_dist2(x1, ax, xx + x1 * x1);
                    f[C_SDMAX] = fmax(f[C_SDMAX], mfs::lorentz_distinf(s1, as));
                    f[C_XDMAX] = fmax(f[C_XDMAX], mfs::lorentz_distinf(x1, ax));
                }
            });
            __syncwarp();
        }
    }
    if constexpr (F32) fold_df_fields<NFC, false>(f, F);
    cta_fields_out<NFC, false>(f, s_red, r.part_col);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_bigcone_resid(const SweepArgs<T> a, const ResidArgs r, int nbig) {
    __shared__ double sh[2 * NWARP];
    const int bq = blockIdx.x;
    const int q = a.big_list[bq];
    const int st = a.soc_start[q], sz = a.soc_size[q];
    Sums<double, 2> acc;
    acc.v[0] = 0.0;
    acc.v[1] = 0.0;
    for (int t = 1 + threadIdx.x; t < sz; t += NT) {
        const double s = r.s_buf[st + t], x = double(a.x[st + t]);
        acc.v[0] += s * s;
        acc.v[1] += x * x;
    }
    acc = block_sum<double, 2>(acc, sh);
    if (threadIdx.x == 0) {
        const double s1 = r.s_buf[st], x1 = double(a.x[st]);
        const double as = sqrt(acc.v[0]), ax = sqrt(acc.v[1]);
        r.part_big[(size_t)B_SDIST2 * nbig + bq] = lorentz_dist2(s1, as, acc.v[0] + s1 * s1);
        r.part_big[(size_t)B_XDIST2 * nbig + bq] = lorentz_dist2(x1, ax, acc.v[1] + x1 * x1);
        r.part_big[(size_t)B_SDMAX * nbig + bq] = mfs::lorentz_distinf(s1, as);
        r.part_big[(size_t)B_XDMAX * nbig + bq] = mfs::lorentz_distinf(x1, ax);
    }
}

// Status block written by the finalizer (matches mfs_residuals_t field order).
enum : int {
    S_RPRIM = 0, S_RDUAL, S_RCONE, S_RGAP, S_KKT, S_POBJ, S_DOBJ,
    S_NRES, S_NB, S_NXDIST, S_NX, S_NSDIST, S_NC, S_NATLC,
    S_IRES, S_IAX, S_IB, S_IATLC, S_IATL, S_IC,
    S_IX, S_IXDIST, S_ISDIST,
    NSTATUS = 23
};

__device__ __forceinline__ double nanmax(double p, double q) {
    return (p > q || p != p) ? p : q;
}

constexpr int NFALL = NFR + NFC + NFB;

// One warp per field folds the per-CTA values in a fixed order; thread 0 then forms the relative
// residuals. Launch with 32 * NFALL threads.
__global__ void __launch_bounds__(32 * NFALL) k_resid_finalize(const double* part_row, int gr, const double* part_col,
                                                               int gc, const double* part_big, int nbig,
                                                               double* status) {
    __shared__ double tot[NFALL];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double* src;
    int cnt;
    bool ismax;
    if (k < NFR) {
        src = part_row + (size_t)k * gr;
        cnt = gr;
        ismax = row_field_is_max(k);
    } else if (k < NFR + NFC) {
        src = part_col + (size_t)(k - NFR) * gc;
        cnt = gc;
        ismax = col_field_is_max(k - NFR);
    } else {
        src = part_big + (size_t)(k - NFR - NFC) * nbig;
        cnt = nbig;
        ismax = big_field_is_max(k - NFR - NFC);
    }
    double acc = 0.0;
    for (int i = lane; i < cnt; i += 32) acc = ismax ? nanmax(acc, src[i]) : acc + src[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const double o = __shfl_down_sync(FULL, acc, d);
        acc = ismax ? nanmax(acc, o) : acc + o;
    }
    if (lane == 0) tot[k] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double* R = tot;
        const double* C = tot + NFR;
        const double* B = tot + NFR + NFC;
        const double nres = sqrt(R[R_RES2]), nb = sqrt(R[R_B2]);
        const double nxd = sqrt(C[C_XDIST2] + B[B_XDIST2]), nsd = sqrt(C[C_SDIST2] + B[B_SDIST2]);
        const double nx = sqrt(C[C_X2]), nc = sqrt(C[C_C2]);
        const double cx = C[C_CX], bl = R[R_BLAM];
        status[S_RPRIM] = nres / (1.0 + nb);
        status[S_RDUAL] = nsd / (1.0 + nc);
        status[S_RCONE] = nxd / (1.0 + nx);
        status[S_RGAP] = fabs(cx + bl) / (1.0 + fabs(cx) + fabs(bl));
        status[S_KKT] = nanmax(nanmax(status[S_RPRIM], status[S_RDUAL]), nanmax(status[S_RCONE], status[S_RGAP]));
        status[S_POBJ] = cx;
        status[S_DOBJ] = -bl;
        status[S_NRES] = nres;
        status[S_NB] = nb;
        status[S_NXDIST] = nxd;
        status[S_NX] = nx;
        status[S_NSDIST] = nsd;
        status[S_NC] = nc;
        status[S_NATLC] = sqrt(C[C_S2]);
        status[S_IRES] = R[R_RESMAX];
        status[S_IAX] = R[R_AXMAX];
        status[S_IB] = R[R_BMAX];
        status[S_IATLC] = C[C_SMAX];
        status[S_IATL] = C[C_ATLMAX];
        status[S_IC] = C[C_CMAX];
        status[S_IX] = C[C_XMAX];
        status[S_IXDIST] = nanmax(C[C_XDMAX], B[B_XDMAX]);
        status[S_ISDIST] = nanmax(C[C_SDMAX], B[B_SDMAX]);
    }
}

// ------------------------------------------------------------------------------------ helpers
template <typename D, typename S>
__global__ void k_convert(D* __restrict__ dst, const S* __restrict__ src, long long count) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x)
        dst[t] = D(src[t]);
}

// out = proj_K(in): the orthant part elementwise; Lorentz cones one thread each (warm start only).
template <typename T>
__global__ void k_proj_orthant(T* __restrict__ out, const double* __restrict__ in, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        out[t] = T(in[t] > 0.0 ? in[t] : 0.0);
}

template <typename T>
__global__ void k_proj_soc(T* __restrict__ out, const double* __restrict__ in, const int* __restrict__ soc_start,
                           const int* __restrict__ soc_size, int nsoc) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsoc) return;
    const int st = soc_start[q], sz = soc_size[q];
    double ss = 0.0;
    for (int t = 1; t < sz; ++t) ss += in[st + t] * in[st + t];
    const double alpha = sqrt(ss), w1 = in[st];
    for (int t = 0; t < sz; ++t) out[st + t] = T(lorentz_coord<double>(in[st + t], t, w1, alpha));
}

}  // namespace mfs
