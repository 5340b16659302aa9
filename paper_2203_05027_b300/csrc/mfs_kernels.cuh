// mfs_kernels.cuh -- the per-iteration sweep and the FP64 residual reductions (sm_103a).
//
// Data layout (built on the host, see mfs_solver.cu): the nonzeros of A are kept twice, in
// column order (CSC: col_ptr, then per-chunk padded row-index/value arrays) and in row order
// (CSR: row_ptr, col-index/value arrays). Columns are grouped into chunks of at most TILE
// nonzeros and CMAX columns; a chunk never splits a Lorentz cone small enough to fit one, and a
// single column longer than TILE is a chunk of its own. Rows are chunked the same way. Each
// chunk's nonzeros start at a multiple of PAD elements in the padded arrays, so one CTA brings
// its whole tile into shared memory with one 1-D bulk copy per array.
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

#include "mfs_device.cuh"

namespace mfs {

template <typename T>
struct SweepArgs {
    // column order
    const int* __restrict__ col_ptr;  // n+1 offsets into the unpadded column order
    const int* __restrict__ cidx;     // padded row indices
    const T* __restrict__ cval;       // padded values
    const int* __restrict__ cj0;      // chunks+1: first column of each column chunk
    const int* __restrict__ ckoff;    // chunks+1: padded offset of each chunk's first nonzero
    const int* __restrict__ cq_lo;    // chunks: first Lorentz cone intersecting the chunk
    const int* __restrict__ cq_hi;    // chunks: one past the last such cone
    // row order
    const int* __restrict__ row_ptr;
    const int* __restrict__ ridx;
    const T* __restrict__ rval;
    const int* __restrict__ ri0;
    const int* __restrict__ rkoff;
    // Lorentz cones, in coordinate order
    const int* __restrict__ soc_start;
    const int* __restrict__ soc_size;
    const unsigned char* __restrict__ soc_big;  // 1: too large to fuse, handled by the big-cone kernel
    const int* __restrict__ big_list;           // indices of the big cones
    // data and iterate
    const T* __restrict__ b;
    const T* __restrict__ c;
    T* x;
    T* z;
    T* del;
    T* lam;
    T* v;
    T mu;
    int* err;
};

template <typename T, typename A, int NV>
struct TileLayout {
    static constexpr int HDR = 128;
    static constexpr int R0 = TILE * (4 + (int)sizeof(T));
    static constexpr int R1 = TILE * NV * (int)sizeof(A);
    static constexpr int R = R0 > R1 ? R0 : R1;
    static constexpr int PTR = HDR + R;
    static constexpr int HEAD = PTR + (CMAX + 8) * 4;
    static constexpr int SCAN = HEAD + TILE / 8;
    static constexpr int EXTRA = SCAN + ((NWARP * NV * (int)sizeof(A) + 127) / 128) * 128;
};

__device__ __forceinline__ void load8(const int* s, int (&o)[8]) {
    int4 u = *reinterpret_cast<const int4*>(s);
    int4 w = *reinterpret_cast<const int4*>(s + 4);
    o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
    o[4] = w.x; o[5] = w.y; o[6] = w.z; o[7] = w.w;
}
__device__ __forceinline__ void load8(const float* s, float (&o)[8]) {
    float4 u = *reinterpret_cast<const float4*>(s);
    float4 w = *reinterpret_cast<const float4*>(s + 4);
    o[0] = u.x; o[1] = u.y; o[2] = u.z; o[3] = u.w;
    o[4] = w.x; o[5] = w.y; o[6] = w.z; o[7] = w.w;
}
__device__ __forceinline__ void load8(const double* s, double (&o)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double2 u = *reinterpret_cast<const double2*>(s + 2 * q);
        o[2 * q] = u.x;
        o[2 * q + 1] = u.y;
    }
}

// Per-segment sums of one chunk of at most TILE nonzeros (segments = the chunk's columns or
// rows). The tile arrives by bulk copy; `pre` runs while it is in flight, `mid` after the first
// barrier. prod(index, value, out[NV]) gives the per-nonzero terms. On return (true) s_end holds,
// at the local position of each segment's last nonzero, that segment's NV sums, and s_ptr the
// local segment offsets. Returns false (CTA must exit) if the bulk copy timed out.
template <typename T, typename A, int NV, typename Prod, typename Pre, typename Mid>
__device__ __forceinline__ bool chunk_sums(const int* __restrict__ gidx, const T* __restrict__ gval, int koff,
                                           int nnz, const int* __restrict__ gptr, int lo, int nseg, int kb,
                                           unsigned char* sm, Prod prod, Pre pre, Mid mid, int* err) {
    using L = TileLayout<T, A, NV>;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
    int* s_ok = reinterpret_cast<int*>(sm + 8);
    int* s_flag = reinterpret_cast<int*>(sm + 16);
    int* s_idx = reinterpret_cast<int*>(sm + L::HDR);
    T* s_val = reinterpret_cast<T*>(sm + L::HDR + TILE * 4);
    A* s_end = reinterpret_cast<A*>(sm + L::HDR);
    int* s_ptr = reinterpret_cast<int*>(sm + L::PTR);
    uint32_t* s_head = reinterpret_cast<uint32_t*>(sm + L::HEAD);
    A* s_scan = reinterpret_cast<A*>(sm + L::SCAN);

    const uint32_t npad = (uint32_t)((nnz + PAD - 1) / PAD * PAD);
    if (threadIdx.x == 0 && npad) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar, npad * (4u + (uint32_t)sizeof(T)));
        bulk_g2s(s_idx, gidx + koff, npad * 4u, bar);
        bulk_g2s(s_val, gval + koff, npad * (uint32_t)sizeof(T), bar);
    }
    for (int t = threadIdx.x; t <= nseg; t += NT) s_ptr[t] = gptr[lo + t] - kb;
    for (int t = threadIdx.x; t < TILE / 32; t += NT) s_head[t] = 0u;
    pre();
    __syncthreads();
    for (int t = threadIdx.x; t < nseg; t += NT) {
        const int st = s_ptr[t];
        if (s_ptr[t + 1] > st) atomicOr(&s_head[st >> 5], 1u << (st & 31));
    }
    mid();
    if (npad) {
        if (!cta_wait_bulk(bar, 0, s_ok, err)) return false;
    } else {
        __syncthreads();
    }

    const int e0 = threadIdx.x * IPT;
    int id[IPT];
    T vl[IPT];
    load8(s_idx + e0, id);
    load8(s_val + e0, vl);
    A p[IPT][NV];
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
        if (e0 + q < nnz) {
            prod(id[q], vl[q], p[q]);
        } else {
#pragma unroll
            for (int t = 0; t < NV; ++t) p[q][t] = A(0);
        }
    }
    const uint32_t hb = (s_head[e0 >> 5] >> (e0 & 31)) & 0xFFu;
    const int en = e0 + IPT;
    const uint32_t nexth = (en < TILE) ? ((s_head[en >> 5] >> (en & 31)) & 1u) : 1u;
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
    // Every thread holds its tile entries in registers before the scan's barrier, so the end
    // sums may overwrite the tile afterwards.
    Sums<A, NV> acc = block_seg_carry<A, NV>(hb != 0u, agg, s_scan, s_flag);
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
            const bool last = (e == nnz - 1) || ((q < IPT - 1) ? ((hb >> (q + 1)) & 1u) : nexth);
            if (last) {
#pragma unroll
                for (int t = 0; t < NV; ++t) s_end[e * NV + t] = acc.v[t];
            }
        }
    }
    __syncthreads();
    return true;
}

// Sums over one segment longer than TILE (a chunk of its own); result valid in thread 0.
template <typename T, typename A, int NV, typename Prod>
__device__ __forceinline__ Sums<A, NV> long_sums(const int* __restrict__ gidx, const T* __restrict__ gval,
                                                 int koff, int nnz, unsigned char* sm, Prod prod) {
    using L = TileLayout<T, A, NV>;
    Sums<A, NV> acc;
#pragma unroll
    for (int t = 0; t < NV; ++t) acc.v[t] = A(0);
    for (int e = threadIdx.x; e < nnz; e += NT) {
        A p[NV];
        prod(gidx[koff + e], gval[koff + e], p);
#pragma unroll
        for (int t = 0; t < NV; ++t) acc.v[t] = acc.v[t] + p[t];
    }
    return block_sum<A, NV>(acc, reinterpret_cast<A*>(sm + L::SCAN));
}

template <typename T>
__device__ __forceinline__ T ldro(const T* p) {
    return __ldg(p);
}

// x-step for one column plus, for an orthant coordinate, the z-step and the delta-update.
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

// ------------------------------------------------------------------------------------ column sweep
template <typename T, bool SOC>
__global__ void __launch_bounds__(NT) k_col_sweep(const SweepArgs<T> a) {
    extern __shared__ __align__(128) unsigned char sm[];
    using L = TileLayout<T, T, 1>;
    const int ch = blockIdx.x;
    const int j0 = a.cj0[ch], j1 = a.cj0[ch + 1], ncol = j1 - j0;
    const int kb = a.col_ptr[j0];
    const int nnz = a.col_ptr[j1] - kb;
    const int koff = a.ckoff[ch];
    const T mu = a.mu;
    const T* __restrict__ v = a.v;
    auto prod = [v](int i, T val, T (&p)[1]) { p[0] = val * ldro(v + i); };

    if (nnz > TILE) {  // one long column
        Sums<T, 1> s = long_sums<T, T, 1>(a.cidx, a.cval, koff, nnz, sm, prod);
        if (threadIdx.x == 0) {
            const int j = j0;
            const T d = T(nnz);
            const T dj = a.del[j];
            const T xn = col_x_update(d, a.x[j], s.v[0], a.z[j], dj, a.c[j], mu);
            a.x[j] = xn;
            const bool in_cone = SOC && (a.cq_hi[ch] > a.cq_lo[ch]);  // then it is a big cone's
            if (!in_cone) {
                const T w = xn - dj / mu;
                const T zn = w > T(0) ? w : T(0);
                a.z[j] = zn;
                a.del[j] = dj + mu * (zn - xn);
            }
        }
        return;
    }

    T* s_x = reinterpret_cast<T*>(sm + L::EXTRA);
    T* s_w = s_x + CMAX;
    T* s_d = s_w + CMAX;
    unsigned char* s_tag = reinterpret_cast<unsigned char*>(s_d + CMAX);

    T px[CPT], pz[CPT], pd[CPT], pc[CPT];
    auto pre = [&]() {
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int jl = threadIdx.x + q * NT;
            if (jl < ncol) {
                px[q] = a.x[j0 + jl];
                pz[q] = a.z[j0 + jl];
                pd[q] = a.del[j0 + jl];
                pc[q] = a.c[j0 + jl];
            }
        }
        if (SOC)
            for (int t = threadIdx.x; t < ncol; t += NT) s_tag[t] = 0;
    };
    auto mid = [&]() {
        if (SOC) {
            __syncthreads();  // s_tag cleared
            for (int q = a.cq_lo[ch] + threadIdx.x; q < a.cq_hi[ch]; q += NT) {
                const int cs = a.soc_start[q], ce = cs + a.soc_size[q];
                const int st = (cs > j0 ? cs : j0) - j0, en = (ce < j1 ? ce : j1) - j0;
                const unsigned char tag = a.soc_big[q] ? 2 : 1;
                for (int t = st; t < en; ++t) s_tag[t] = tag;
            }
        }
    };
    if (!chunk_sums<T, T, 1>(a.cidx, a.cval, koff, nnz, a.col_ptr, j0, ncol, kb, sm, prod, pre, mid, a.err))
        return;
    const T* s_end = reinterpret_cast<const T*>(sm + L::HDR);
    const int* s_ptr = reinterpret_cast<const int*>(sm + L::PTR);
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int jl = threadIdx.x + q * NT;
        if (jl < ncol) {
            const int st = s_ptr[jl], en = s_ptr[jl + 1];
            const T atv = (en > st) ? s_end[en - 1] : T(0);
            const T xn = col_x_update(T(en - st), px[q], atv, pz[q], pd[q], pc[q], mu);
            const int j = j0 + jl;
            a.x[j] = xn;
            const unsigned char tag = SOC ? s_tag[jl] : 0;
            if (tag == 0) {
                const T w = xn - pd[q] / mu;
                const T zn = w > T(0) ? w : T(0);
                a.z[j] = zn;
                a.del[j] = pd[q] + mu * (zn - xn);
            } else if (tag == 1) {
                s_x[jl] = xn;
                s_w[jl] = xn - pd[q] / mu;
                s_d[jl] = pd[q];
            }
        }
    }
    if (SOC) {
        __syncthreads();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int q = a.cq_lo[ch] + warp; q < a.cq_hi[ch]; q += NWARP) {
            if (a.soc_big[q]) continue;
            const int st = a.soc_start[q] - j0, sz = a.soc_size[q];
            T ss = T(0);
            for (int t = 1 + lane; t < sz; t += 32) ss += s_w[st + t] * s_w[st + t];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, d);
            const T alpha = sqrt(ss);
            const T w1 = s_w[st];
            for (int t = lane; t < sz; t += 32) {
                const T zt = lorentz_coord(s_w[st + t], t, w1, alpha);
                a.z[j0 + st + t] = zt;
                a.del[j0 + st + t] = s_d[st + t] + mu * (zt - s_x[st + t]);
            }
        }
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
// MODE 0: iteration (lambda and v updated). MODE 1: warm start (v from x and a given lambda).
template <typename T, int MODE>
__global__ void __launch_bounds__(NT) k_row_sweep(const SweepArgs<T> a) {
    extern __shared__ __align__(128) unsigned char sm[];
    using L = TileLayout<T, T, 2>;
    const int ch = blockIdx.x;
    const int i0 = a.ri0[ch], i1 = a.ri0[ch + 1], nrow = i1 - i0;
    const int kb = a.row_ptr[i0];
    const int nnz = a.row_ptr[i1] - kb;
    const int koff = a.rkoff[ch];
    const T mu = a.mu;
    const T* __restrict__ x = a.x;
    auto prod = [x](int j, T val, T (&p)[2]) {
        p[0] = val * ldro(x + j);
        p[1] = val * val;
    };
    if (nnz > TILE) {
        Sums<T, 2> s = long_sums<T, T, 2>(a.ridx, a.rval, koff, nnz, sm, prod);
        if (threadIdx.x == 0) {
            const T rho = (a.b[i0] - s.v[0]) / (T(1) + s.v[1]);
            const T l = a.lam[i0];
            if (MODE == 0) {
                const T ln = l - mu * rho;
                a.lam[i0] = ln;
                a.v[i0] = rho - ln / mu;
            } else {
                a.v[i0] = rho - l / mu;
            }
        }
        return;
    }
    T pb[CPT], pl[CPT];
    auto pre = [&]() {
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int il = threadIdx.x + q * NT;
            if (il < nrow) {
                pb[q] = a.b[i0 + il];
                pl[q] = a.lam[i0 + il];
            }
        }
    };
    auto mid = []() {};
    if (!chunk_sums<T, T, 2>(a.ridx, a.rval, koff, nnz, a.row_ptr, i0, nrow, kb, sm, prod, pre, mid, a.err))
        return;
    const T* s_end = reinterpret_cast<const T*>(sm + L::HDR);
    const int* s_ptr = reinterpret_cast<const int*>(sm + L::PTR);
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int il = threadIdx.x + q * NT;
        if (il < nrow) {
            const int st = s_ptr[il], en = s_ptr[il + 1];
            const T ax = (en > st) ? s_end[2 * (en - 1)] : T(0);
            const T r = (en > st) ? s_end[2 * (en - 1) + 1] : T(0);
            const T rho = (pb[q] - ax) / (T(1) + r);
            const int i = i0 + il;
            if (MODE == 0) {
                const T ln = pl[q] - mu * rho;
                a.lam[i] = ln;
                a.v[i] = rho - ln / mu;
            } else {
                a.v[i] = rho - pl[q] / mu;
            }
        }
    }
}

// ------------------------------------------------------------------------------------ residuals
// Partial-sum fields, one row of NF doubles per CTA.
enum : int {
    F_RES2 = 0, F_RESMAX, F_AXMAX, F_B2, F_BMAX, F_BLAM,
    F_S2, F_SMAX, F_ATLMAX, F_C2, F_CMAX, F_CX, F_X2, F_SDIST2, F_XDIST2,
    NF = 16
};

__device__ __forceinline__ bool field_is_max(int f) {
    return f == F_RESMAX || f == F_AXMAX || f == F_BMAX || f == F_SMAX || f == F_ATLMAX || f == F_CMAX;
}

// Squared distance of w to one Lorentz cone, given w_1 and alpha = ||w_{2..}||
// (w - P(w) is 0, w, or has norm^2 (alpha - w_1)^2 / 2 in the three cases of eq. proj).
__device__ __forceinline__ double lorentz_dist2(double w1, double alpha, double wnorm2) {
    if (alpha <= -w1) return wnorm2;
    if (alpha <= w1) return 0.0;
    const double g = alpha - w1;
    return 0.5 * g * g;
}

__device__ __forceinline__ void write_partials(double* out, double (&f)[NF], double* sh) {
    for (int k = 0; k < NF; ++k) {
        double r;
        if (field_is_max(k)) {
            r = block_max(f[k], sh);
        } else {
            Sums<double, 1> s;
            s.v[0] = f[k];
            r = block_sum<double, 1>(s, sh).v[0];
        }
        if (threadIdx.x == 0) out[k] = r;
    }
}

struct ResidArgs {
    double* part_row;  // row chunks x NF
    double* part_col;  // column chunks x NF
    double* part_big;  // big cones x NF
    double* s_buf;     // n: c + A^T lambda (FP64), written for big-cone columns (all if write_all_s)
    int write_all_s;
};

template <typename T>
__global__ void __launch_bounds__(NT) k_row_resid(const SweepArgs<T> a, const ResidArgs r) {
    extern __shared__ __align__(128) unsigned char sm[];
    using L = TileLayout<T, double, 1>;
    const int ch = blockIdx.x;
    const int i0 = a.ri0[ch], i1 = a.ri0[ch + 1], nrow = i1 - i0;
    const int kb = a.row_ptr[i0];
    const int nnz = a.row_ptr[i1] - kb;
    const int koff = a.rkoff[ch];
    const T* __restrict__ x = a.x;
    auto prod = [x](int j, T val, double (&p)[1]) { p[0] = double(val) * double(ldro(x + j)); };
    double f[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) f[k] = 0.0;
    double* shred = reinterpret_cast<double*>(sm + L::EXTRA);
    if (nnz > TILE) {
        Sums<double, 1> s = long_sums<T, double, 1>(a.ridx, a.rval, koff, nnz, sm, prod);
        if (threadIdx.x == 0) {
            const double bi = double(a.b[i0]);
            const double res = s.v[0] - bi;
            f[F_RES2] = res * res;
            f[F_RESMAX] = fabs(res);
            f[F_AXMAX] = fabs(s.v[0]);
            f[F_B2] = bi * bi;
            f[F_BMAX] = fabs(bi);
            f[F_BLAM] = bi * double(a.lam[i0]);
        }
        write_partials(r.part_row + (size_t)ch * NF, f, shred);
        return;
    }
    auto none = []() {};
    if (!chunk_sums<T, double, 1>(a.ridx, a.rval, koff, nnz, a.row_ptr, i0, nrow, kb, sm, prod, none, none,
                                  a.err))
        return;
    const double* s_end = reinterpret_cast<const double*>(sm + L::HDR);
    const int* s_ptr = reinterpret_cast<const int*>(sm + L::PTR);
    for (int il = threadIdx.x; il < nrow; il += NT) {
        const int st = s_ptr[il], en = s_ptr[il + 1];
        const double ax = (en > st) ? s_end[en - 1] : 0.0;
        const double bi = double(a.b[i0 + il]);
        const double res = ax - bi;
        f[F_RES2] += res * res;
        f[F_RESMAX] = fmax(f[F_RESMAX], fabs(res));
        f[F_AXMAX] = fmax(f[F_AXMAX], fabs(ax));
        f[F_B2] += bi * bi;
        f[F_BMAX] = fmax(f[F_BMAX], fabs(bi));
        f[F_BLAM] += bi * double(a.lam[i0 + il]);
    }
    write_partials(r.part_row + (size_t)ch * NF, f, shred);
}

template <typename T, bool SOC>
__global__ void __launch_bounds__(NT) k_col_resid(const SweepArgs<T> a, const ResidArgs r) {
    extern __shared__ __align__(128) unsigned char sm[];
    using L = TileLayout<T, double, 1>;
    const int ch = blockIdx.x;
    const int j0 = a.cj0[ch], j1 = a.cj0[ch + 1], ncol = j1 - j0;
    const int kb = a.col_ptr[j0];
    const int nnz = a.col_ptr[j1] - kb;
    const int koff = a.ckoff[ch];
    const T* __restrict__ lam = a.lam;
    auto prod = [lam](int i, T val, double (&p)[1]) { p[0] = double(val) * double(ldro(lam + i)); };
    double f[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) f[k] = 0.0;
    double* shred = reinterpret_cast<double*>(sm + L::EXTRA);
    double* s_s = shred + 2 * NWARP;  // CMAX
    double* s_xv = s_s + CMAX;        // CMAX
    unsigned char* s_tag = reinterpret_cast<unsigned char*>(s_xv + CMAX);

    // per-column work shared by the two paths; tag 0 orthant, 1 small cone, 2 big cone
    auto column = [&](int jl, double atl, unsigned char tag) {
        const int j = j0 + jl;
        const double cj = double(a.c[j]), xj = double(a.x[j]);
        const double s = cj + atl;
        f[F_S2] += s * s;
        f[F_SMAX] = fmax(f[F_SMAX], fabs(s));
        f[F_ATLMAX] = fmax(f[F_ATLMAX], fabs(atl));
        f[F_C2] += cj * cj;
        f[F_CMAX] = fmax(f[F_CMAX], fabs(cj));
        f[F_CX] += cj * xj;
        f[F_X2] += xj * xj;
        if (tag == 0) {
            const double sn = s < 0.0 ? s : 0.0, xn = xj < 0.0 ? xj : 0.0;
            f[F_SDIST2] += sn * sn;
            f[F_XDIST2] += xn * xn;
        } else if (tag == 1) {
            s_s[jl] = s;
            s_xv[jl] = xj;
        }
        if (tag == 2 || r.write_all_s) r.s_buf[j] = s;
    };

    if (nnz > TILE) {
        Sums<double, 1> s = long_sums<T, double, 1>(a.cidx, a.cval, koff, nnz, sm, prod);
        if (threadIdx.x == 0) {
            const bool in_cone = SOC && (a.cq_hi[ch] > a.cq_lo[ch]);
            column(0, s.v[0], in_cone ? 2 : 0);
        }
        write_partials(r.part_col + (size_t)ch * NF, f, shred);
        return;
    }
    auto pre = [&]() {
        if (SOC)
            for (int t = threadIdx.x; t < ncol; t += NT) s_tag[t] = 0;
    };
    auto mid = [&]() {
        if (SOC) {
            __syncthreads();
            for (int q = a.cq_lo[ch] + threadIdx.x; q < a.cq_hi[ch]; q += NT) {
                const int cs = a.soc_start[q], ce = cs + a.soc_size[q];
                const int st = (cs > j0 ? cs : j0) - j0, en = (ce < j1 ? ce : j1) - j0;
                const unsigned char tag = a.soc_big[q] ? 2 : 1;
                for (int t = st; t < en; ++t) s_tag[t] = tag;
            }
        }
    };
    if (!chunk_sums<T, double, 1>(a.cidx, a.cval, koff, nnz, a.col_ptr, j0, ncol, kb, sm, prod, pre, mid, a.err))
        return;
    const double* s_end = reinterpret_cast<const double*>(sm + L::HDR);
    const int* s_ptr = reinterpret_cast<const int*>(sm + L::PTR);
    for (int jl = threadIdx.x; jl < ncol; jl += NT) {
        const int st = s_ptr[jl], en = s_ptr[jl + 1];
        column(jl, (en > st) ? s_end[en - 1] : 0.0, SOC ? s_tag[jl] : 0);
    }
    if (SOC) {
        __syncthreads();
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        double dsum_s = 0.0, dsum_x = 0.0;
        for (int q = a.cq_lo[ch] + warp; q < a.cq_hi[ch]; q += NWARP) {
            if (a.soc_big[q]) continue;
            const int st = a.soc_start[q] - j0, sz = a.soc_size[q];
            double ss = 0.0, xx = 0.0;
            for (int t = 1 + lane; t < sz; t += 32) {
                ss += s_s[st + t] * s_s[st + t];
                xx += s_xv[st + t] * s_xv[st + t];
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                ss += __shfl_xor_sync(0xffffffffu, ss, d);
                xx += __shfl_xor_sync(0xffffffffu, xx, d);
            }
            if (lane == 0) {
                const double s1 = s_s[st], x1 = s_xv[st];
                dsum_s += lorentz_dist2(s1, sqrt(ss), ss + s1 * s1);
                dsum_x += lorentz_dist2(x1, sqrt(xx), xx + x1 * x1);
            }
        }
        f[F_SDIST2] += dsum_s;
        f[F_XDIST2] += dsum_x;
    }
    write_partials(r.part_col + (size_t)ch * NF, f, shred);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_bigcone_resid(const SweepArgs<T> a, const ResidArgs r) {
    __shared__ double sh[2 * NWARP];
    const int b = blockIdx.x;
    const int q = a.big_list[b];
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
        double* out = r.part_big + (size_t)b * NF;
        for (int k = 0; k < NF; ++k) out[k] = 0.0;
        const double s1 = r.s_buf[st], x1 = double(a.x[st]);
        out[F_SDIST2] = lorentz_dist2(s1, sqrt(acc.v[0]), acc.v[0] + s1 * s1);
        out[F_XDIST2] = lorentz_dist2(x1, sqrt(acc.v[1]), acc.v[1] + x1 * x1);
    }
}

// Status block written by the finalizer (matches mfs_residuals_t field order).
enum : int {
    S_RPRIM = 0, S_RDUAL, S_RCONE, S_RGAP, S_KKT, S_POBJ, S_DOBJ,
    S_NRES, S_NB, S_NXDIST, S_NX, S_NSDIST, S_NC, S_NATLC,
    S_IRES, S_IAX, S_IB, S_IATLC, S_IATL, S_IC,
    NSTATUS = 20
};

__device__ __forceinline__ double nanmax(double p, double q) {
    return (p > q || p != p) ? p : q;
}

__global__ void __launch_bounds__(NT) k_resid_finalize(const double* part_row, int nrow_parts,
                                                       const double* part_col, int ncol_parts,
                                                       const double* part_big, int nbig, double* status) {
    __shared__ double sh[NWARP];
    __shared__ double tot[NF];
    for (int k = 0; k < NF; ++k) {
        const bool ismax = field_is_max(k);
        double acc = 0.0;
        for (int i = threadIdx.x; i < nrow_parts; i += NT) {
            const double v = part_row[(size_t)i * NF + k];
            acc = ismax ? nanmax(acc, v) : acc + v;
        }
        for (int i = threadIdx.x; i < ncol_parts; i += NT) {
            const double v = part_col[(size_t)i * NF + k];
            acc = ismax ? nanmax(acc, v) : acc + v;
        }
        for (int i = threadIdx.x; i < nbig; i += NT) {
            const double v = part_big[(size_t)i * NF + k];
            acc = ismax ? nanmax(acc, v) : acc + v;
        }
        double r;
        if (ismax) {
            r = block_max(acc, sh);
        } else {
            Sums<double, 1> s;
            s.v[0] = acc;
            r = block_sum<double, 1>(s, sh).v[0];
        }
        if (threadIdx.x == 0) tot[k] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double nres = sqrt(tot[F_RES2]), nb = sqrt(tot[F_B2]), nxd = sqrt(tot[F_XDIST2]);
        const double nx = sqrt(tot[F_X2]), nsd = sqrt(tot[F_SDIST2]), nc = sqrt(tot[F_C2]);
        const double cx = tot[F_CX], bl = tot[F_BLAM];
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
        status[S_NATLC] = sqrt(tot[F_S2]);
        status[S_IRES] = tot[F_RESMAX];
        status[S_IAX] = tot[F_AXMAX];
        status[S_IB] = tot[F_BMAX];
        status[S_IATLC] = tot[F_SMAX];
        status[S_IATL] = tot[F_ATLMAX];
        status[S_IC] = tot[F_CMAX];
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
