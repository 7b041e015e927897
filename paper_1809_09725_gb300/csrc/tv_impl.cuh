// tv_impl.cuh -- 4D total-variation kernels on the synthesised frames.
//
// The regulariser of Eq. (TV1) acts on frames f(x, t_l) = sum_j phi_j(t_l)
// u_j(x), l = 0..nt-1 (Sec. 4, Eq. discrt).  With D = nabla_{lambda2} o PhiF
// (forward differences, zero across the last index of each dimension,
// lambda2 on the time component) the kernels compute, per voxel, without
// ever storing the frames:
//   D u      : nabla along x,y,z of sum_j PhiF[l][j] u_j  =  sum_j PhiF[l][j] (u_j(x+e) - u_j(x));
//              time part lambda2 sum_j (PhiF[l+1][j] - PhiF[l][j]) u_j(x)
//   D^T p    : PhiF^T (-div p)  (Sec. 3, K_2^* = -div_{lambda2})
//   D^T D x  : G (L_s x) + lambda2^2 Lt x with G = PhiF^T PhiF and
//              Lt = PhiF^T L_t PhiF (m x m), L_s / L_t the Neumann Laplacians
//              (the composition of the two stencils, exact up to rounding)
//   ADMM shrink/dual update, CP projection and primal update (Sec. 3, Fig. 2)
// All are HBM bound; each thread owns whole voxels (all m coefficients and
// all nt frames).  The volume is walked in bands of rows (band_voxel) by
// grids of resident blocks (tv_grid), so neighbours come through L1/L2; D^T D
// on FP32 rows of 4, 8 or 16 floats marches tiles up z with the rows staged in
// shared memory (lap_tile_kernel).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#pragma once
#include "dr_device.cuh"

namespace dr {

template <typename T>
struct V4;
template <>
struct V4<float> {
    typedef float4 type;
};
struct D4 {
    double x, y, z, w;
};
template <>
struct V4<double> {
    typedef D4 type;
};

template <typename T>
__device__ __forceinline__ typename V4<T>::type ld4(const T *p);
template <>
__device__ __forceinline__ float4 ld4<float>(const float *p) { return *reinterpret_cast<const float4 *>(p); }
template <>
__device__ __forceinline__ D4 ld4<double>(const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    return D4{a.x, a.y, b.x, b.y};
}
template <typename T, typename V>
__device__ __forceinline__ void st4(T *p, V v);
template <>
__device__ __forceinline__ void st4<float, float4>(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
template <>
__device__ __forceinline__ void st4<double, D4>(double *p, D4 v) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v.x, v.y);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v.z, v.w);
}

// Dual fields stored as F: the compute type, or bf16 for plans that keep the
// solver's dual fields in bf16 (arithmetic stays in T; one rounding to the
// nearest bf16 per store).
template <typename T, typename F>
struct FieldIO {
    static __device__ __forceinline__ typename V4<T>::type ld(const T *p) { return ld4<T>(p); }
    static __device__ __forceinline__ void st(T *p, typename V4<T>::type v) { st4<T>(p, v); }
    static __device__ __forceinline__ T ld1(const T *p) { return *p; }
};
template <>
struct FieldIO<float, bf16> {
    static __device__ __forceinline__ float4 ld(const bf16 *p) {
        const uint2 a = *reinterpret_cast<const uint2 *>(p);
        return make_float4(__uint_as_float(a.x << 16), __uint_as_float(a.x & 0xffff0000u),
                           __uint_as_float(a.y << 16), __uint_as_float(a.y & 0xffff0000u));
    }
    static __device__ __forceinline__ void st(bf16 *p, float4 v) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 o;
        o.x = *reinterpret_cast<const unsigned *>(&a);
        o.y = *reinterpret_cast<const unsigned *>(&b);
        *reinterpret_cast<uint2 *>(p) = o;
    }
    static __device__ __forceinline__ float ld1(const bf16 *p) { return __bfloat162float(*p); }
};

// zlo / zhi: the slice below local z = 0 / above local z = nz-1 exists in
// memory (a halo of a slab of a larger volume), so the z differences there
// are interior ones instead of the Neumann boundary.  band: rows of y per
// band of the traversal order (band_voxel).
struct Geo {
    int nx, ny, nz, m, nt;
    int zlo, zhi;
    int band;
};

// Traversal order of the stencil kernels.  The volume is cut into bands of
// g.band rows of y; a band is walked slice by slice (its rows at one z, then
// the same rows at z+1), and the bands follow one another.  Step w of the walk
// is voxel v = (z ny + y) nx + x.  Consecutive steps are consecutive x (a
// warp's loads stay coalesced), and the z neighbours of a voxel are visited
// g.band rows before and after it, so they are still in L2 when a stencil
// reads them; walking the whole slice before the next one (g.band = ny) puts a
// full slice between them, more than L2 holds on large volumes.
__device__ __forceinline__ size_t band_voxel(size_t w, const Geo &g, int &x, int &y, int &z) {
    x = (int)(w % g.nx);
    const size_t r = w / g.nx;  // row of the walk
    const size_t full = (size_t)(g.ny / g.band) * g.band;  // rows of y in full bands
    const size_t rf = full * g.nz;                          // walk rows inside full bands
    if (r < rf) {
        const size_t per = (size_t)g.band * g.nz;
        const size_t b = r / per, q = r % per;
        z = (int)(q / g.band);
        y = (int)(b * g.band + q % g.band);
    } else {
        const int h = g.ny - (int)full;  // rows of the last, partial band
        const size_t q = r - rf;
        z = (int)(q / h);
        y = (int)(full + q % h);
    }
    return ((size_t)z * g.ny + y) * g.nx + x;
}

// 4-vector fields on frames (D u, the duals) are stored frame-major within
// each slice, [nz][nt][ny][nx][4]: the threads of a warp (consecutive voxels)
// read or write one frame as one contiguous run of 16-byte vectors, and a
// z-slab of slices is still one contiguous block.  field_base is the offset
// of voxel v's frame 0; frame l adds l * frame_stride.
__device__ __forceinline__ size_t field_base(size_t v, int z, const Geo &g) {
    return (v + (size_t)z * (g.nt - 1) * g.nx * g.ny) * 4;
}
__device__ __forceinline__ size_t frame_stride(const Geo &g) { return (size_t)g.nx * g.ny * 4; }

// Shared-memory copies of PhiF / dPhiF ([nt][M]) and G / Lt ([M][M]).
template <typename T, int M>
__device__ __forceinline__ void load_tables(T *sm, const T *PhiF, const T *dPhiF, const T *G, const T *Lt, int nt,
                                            bool want_gl) {
    const int n1 = nt * M;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        sm[i] = PhiF[i];
        sm[n1 + i] = dPhiF[i];
    }
    if (want_gl)
        for (int i = threadIdx.x; i < M * M; i += blockDim.x) {
            sm[2 * n1 + i] = G[i];
            sm[2 * n1 + M * M + i] = Lt[i];
        }
    __syncthreads();
}

// Spatial forward differences of the coefficients at voxel v (Neumann).
template <typename T, typename S, int M>
__device__ __forceinline__ void coeff_diffs(const S *__restrict__ u, size_t v, int x, int y, int z, const Geo &g,
                                            T (&uc)[M], T (&ex)[M], T (&ey)[M], T (&ez)[M]) {
    load_coeffs<T, S, M>(u + v * g.m, g.m, uc);
    if (x + 1 < g.nx) {
        load_coeffs<T, S, M>(u + (v + 1) * g.m, g.m, ex);
#pragma unroll
        for (int j = 0; j < M; ++j) ex[j] -= uc[j];
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) ex[j] = T(0);
    }
    if (y + 1 < g.ny) {
        load_coeffs<T, S, M>(u + (v + g.nx) * g.m, g.m, ey);
#pragma unroll
        for (int j = 0; j < M; ++j) ey[j] -= uc[j];
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) ey[j] = T(0);
    }
    if (z + 1 < g.nz || g.zhi) {
        load_coeffs<T, S, M>(u + (v + (size_t)g.nx * g.ny) * g.m, g.m, ez);
#pragma unroll
        for (int j = 0; j < M; ++j) ez[j] -= uc[j];
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) ez[j] = T(0);
    }
}

// Spatial components of (D u)(x, t_l) from the coefficient differences.
template <typename T, int M>
__device__ __forceinline__ void grad_frame(const T *sm, int l, const T (&ex)[M], const T (&ey)[M],
                                           const T (&ez)[M], T &gx, T &gy, T &gz) {
    const T *ph = sm + l * M;
    gx = gy = gz = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j) {
        gx = fma(ph[j], ex[j], gx);
        gy = fma(ph[j], ey[j], gy);
        gz = fma(ph[j], ez[j], gz);
    }
}

// Time component lambda2 sum_j (PhiF[l+1][j] - PhiF[l][j]) u_j (zero for the last frame).
template <typename T, int M>
__device__ __forceinline__ T dt_frame(const T *dph_l, T lambda2, const T (&uc)[M]) {
    T s = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j) s = fma(dph_l[j], uc[j], s);
    return lambda2 * s;
}

// ---------------------------------------------------------------------------
// p = D u
// ---------------------------------------------------------------------------
template <typename T, typename S, int M>
__global__ void __launch_bounds__(kRedThreads)
    grad_kernel(const S *__restrict__ u, T *__restrict__ p, const T *PhiF, const T *dPhiF, Geo g, T lambda2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    load_tables<T, M>(sm, PhiF, dPhiF, nullptr, nullptr, g.nt, false);
    const T *dph = sm + g.nt * M;
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < nv; it += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        const size_t v = band_voxel(it, g, x, y, z);
        T uc[M], ex[M], ey[M], ez[M];
        coeff_diffs<T, S, M>(u, v, x, y, z, g, uc, ex, ey, ez);
        const size_t fb = field_base(v, z, g), fs = frame_stride(g);
        for (int l = 0; l < g.nt; ++l) {
            T gx, gy, gz, gt;
            grad_frame<T, M>(sm, l, ex, ey, ez, gx, gy, gz);
            gt = dt_frame<T, M>(dph + l * M, lambda2, uc);
            typename V4<T>::type o;
            o.x = gx;
            o.y = gy;
            o.z = gz;
            o.w = gt;
            st4<T>(p + fb + l * fs, o);
        }
    }
}

// (D^T p)_j at voxel v (Neumann-matched backward differences, then PhiF^T).
// PhiF and dPhiF ([nt][M]) as a kernel parameter for FP32 D^T when nt M is at
// most kFrameTabMax: the rows of frame l are then read through the constant
// cache instead of shared memory (whose loads share the L1 pipe with the
// field's).
constexpr int kFrameTabMax = 448;
template <typename T>
struct FrameTab {
    static constexpr int kMax = sizeof(T) == 4 ? kFrameTabMax : 1;
    T ph[kMax];
    T dph[kMax];
};

template <typename T, int M, typename F = T, bool CT = false>
__device__ __forceinline__ void gradT_voxel(const F *__restrict__ p, size_t v, int x, int y, int z, const Geo &g,
                                            const T *sm, T lambda2, T (&outj)[M],
                                            const FrameTab<T> *ft = nullptr) {
    const T *dph = sm + g.nt * M;
#pragma unroll
    for (int j = 0; j < M; ++j) outj[j] = T(0);
    const size_t fs = frame_stride(g);
    const size_t sx = 4, sy = (size_t)g.nx * 4, sz = (size_t)g.nt * fs;
    const F *pv = p + field_base(v, z, g);
    const bool hx = x + 1 < g.nx, lx = x > 0, hy = y + 1 < g.ny, ly = y > 0;
    const bool hz = z + 1 < g.nz || g.zhi, lz = z > 0 || g.zlo;
    // frames in groups of FG: all their loads are issued before the sums
    // (more bytes in flight per thread); the sums keep the frame order
    constexpr int FG = 4;
    for (int l0 = 0; l0 < g.nt; l0 += FG) {
        typename V4<T>::type q[FG];
        T nbx[FG], nby[FG], nbz[FG];
#pragma unroll
        for (int f = 0; f < FG; ++f) {
            const int l = l0 + f;
            if (l < g.nt) {
                q[f] = FieldIO<T, F>::ld(pv + l * fs);
                nbx[f] = lx ? FieldIO<T, F>::ld1(pv - sx + l * fs + 0) : T(0);
                nby[f] = ly ? FieldIO<T, F>::ld1(pv - sy + l * fs + 1) : T(0);
                nbz[f] = lz ? FieldIO<T, F>::ld1(pv - sz + l * fs + 2) : T(0);
            }
        }
#pragma unroll
        for (int f = 0; f < FG; ++f) {
            const int l = l0 + f;
            if (l >= g.nt) break;
            T s = T(0);
            if (hx) s -= q[f].x;
            if (lx) s += nbx[f];
            if (hy) s -= q[f].y;
            if (ly) s += nby[f];
            if (hz) s -= q[f].z;
            if (lz) s += nbz[f];
            const T qt = lambda2 * q[f].w;
            if constexpr (CT) {
                const T *ph = ft->ph + l * M;
                const T *dp = ft->dph + l * M;
#pragma unroll
                for (int j = 0; j < M; ++j) outj[j] = fma(ph[j], s, fma(dp[j], qt, outj[j]));
            } else {
                const T *ph = sm + l * M;
                const T *dp = dph + l * M;
#pragma unroll
                for (int j = 0; j < M; ++j) outj[j] = fma(ph[j], s, fma(dp[j], qt, outj[j]));
            }
        }
    }
}

// u = beta u + alpha D^T p
// Resident CTAs per SM asked of the FP32 instantiations: four at m <= 8
// (64 registers), three at m = 16 (85), two at m = 32.
__host__ __device__ constexpr int gradT_min_blocks(int M, int T_bytes) {
    return T_bytes == 4 ? (M <= 8 ? 4 : (M == 16 ? 3 : 2)) : 1;
}

template <typename T, typename S, int M, typename F = T, bool CT = false>
__global__ void __launch_bounds__(kRedThreads, gradT_min_blocks(M, sizeof(T)))
    gradT_kernel(const F *__restrict__ p, S *__restrict__ u_s, T *__restrict__ u_c, const T *PhiF, const T *dPhiF,
                 Geo g, T lambda2, T alpha, T beta, const __grid_constant__ FrameTab<T> ft) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    if constexpr (!CT) load_tables<T, M>(sm, PhiF, dPhiF, nullptr, nullptr, g.nt, false);
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < nv; it += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        const size_t v = band_voxel(it, g, x, y, z);
        T o[M];
        gradT_voxel<T, M, F, CT>(p, v, x, y, z, g, sm, lambda2, o, &ft);
        if (u_c) {
            // compute-typed row: vector loads and stores
            T ov[M];
#pragma unroll
            for (int j = 0; j < M; ++j) o[j] = alpha * o[j];
            if (beta != T(0)) {
                load_row<T, M>(u_c + v * g.m, g.m, ov);
#pragma unroll
                for (int j = 0; j < M; ++j) o[j] += beta * ov[j];
            }
            store_row<T, M>(u_c + v * g.m, g.m, o);
            continue;
        }
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j >= g.m) break;
            const size_t i = v * g.m + j;
            T r = alpha * o[j];
            if (beta != T(0)) r += beta * ldc<T>(u_s + i);
            stc<T>(u_s + i, r);
        }
    }
}

// ---------------------------------------------------------------------------
// ADMM prox: v = Du + mu/rho; psi = shrink(v, lambda1/rho); mu += rho (Du - psi);
// w = psi - mu/rho.  Reduces sum |Du| and ||Du - psi||^2.
// obj: destination row (tv, primal^2); when use_iter the row is obj + 3*iter + 1.
// ---------------------------------------------------------------------------
// prox keeps a group of frames' duals in registers besides the coefficient
// differences: three CTAs per SM (85 registers) at m <= 8, two (128) at
// m = 16, where the group is four frames (64 bytes of loads in flight per
// thread)
__host__ __device__ constexpr int prox_min_blocks(int M, int T_bytes) {
    return T_bytes == 4 ? (M <= 8 ? 3 : (M == 16 ? 2 : 1)) : 1;
}

template <typename T, typename S, int M, typename F = T>
__global__ void __launch_bounds__(kRedThreads, prox_min_blocks(M, sizeof(T)))
    prox_kernel(const S *__restrict__ u, F *__restrict__ mu, F *__restrict__ w, const T *PhiF, const T *dPhiF, Geo g,
                T rho, T lambda1, T lambda2, double *partials, unsigned *counter, DevScalars *scal, double *obj,
                int use_iter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    load_tables<T, M>(sm, PhiF, dPhiF, nullptr, nullptr, g.nt, false);
    const T *dph = sm + g.nt * M;
    const T kappa = lambda1 / rho, irho = T(1) / rho;
    PartialSum<T> acc_tv, acc_pr;
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < nv; it += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        const size_t v = band_voxel(it, g, x, y, z);
        T uc[M], ex[M], ey[M], ez[M];
        coeff_diffs<T, S, M>(u, v, x, y, z, g, uc, ex, ey, ez);
        // frames in groups of FG: the group's dual loads are issued first (more
        // bytes in flight per thread); the frames are then processed in order
        constexpr int FG = (M == 16 && sizeof(T) == 4) ? 4 : 2;
        const size_t fb = field_base(v, z, g), fs = frame_stride(g);
        for (int l0 = 0; l0 < g.nt; l0 += FG) {
            typename V4<T>::type mg[FG];
#pragma unroll
            for (int h = 0; h < FG; ++h)
                if (l0 + h < g.nt) mg[h] = FieldIO<T, F>::ld(mu + fb + (l0 + h) * fs);
#pragma unroll
            for (int h = 0; h < FG; ++h) {
                const int l = l0 + h;
                if (l >= g.nt) break;
                T d[4];
                grad_frame<T, M>(sm, l, ex, ey, ez, d[0], d[1], d[2]);
                d[3] = dt_frame<T, M>(dph + l * M, lambda2, uc);
                const size_t o = fb + l * fs;
                const T mv[4] = {mg[h].x, mg[h].y, mg[h].z, mg[h].w};
                T vv[4];
                T n2 = T(0), dn2 = T(0);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    vv[c] = d[c] + mv[c] * irho;
                    n2 += vv[c] * vv[c];
                    dn2 += d[c] * d[c];
                }
                const T n = sqrt(n2);
                const T f = (n > T(0)) ? fmax(T(0), T(1) - kappa / n) : T(0);
                T mn[4], wn[4];
                T pr = T(0);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const T psi = vv[c] * f;
                    const T r = d[c] - psi;
                    pr = fma(r, r, pr);
                    mn[c] = mv[c] + rho * r;
                    wn[c] = psi - mn[c] * irho;
                }
                // per-frame terms in the compute type; FP64 only across threads
                acc_tv.add(sqrt(dn2));
                acc_pr.add(pr);
                typename V4<T>::type a, b;
                a.x = mn[0]; a.y = mn[1]; a.z = mn[2]; a.w = mn[3];
                b.x = wn[0]; b.y = wn[1]; b.z = wn[2]; b.w = wn[3];
                FieldIO<T, F>::st(mu + o, a);
                FieldIO<T, F>::st(w + o, b);
            }
        }
    }
    double vals[2] = {acc_tv.value(), acc_pr.value()}, tot[2];
    if (block_reduce_last<2>(vals, partials, counter, tot)) {
        double *row = use_iter ? obj + 3 * (size_t)scal->iter : obj;
        if (row) {
            row[1] = tot[0];
            row[2] = tot[1];
        } else {
            scal->acc1 = tot[0];
            scal->acc2 = tot[1];
        }
    }
}

// ---------------------------------------------------------------------------
// out = beta out + alpha (G L_s x + lambda2^2 Lt x), G L_s + lambda2^2 Lt being
// D^T D.  mode 0: reduce <x, out> into scal->pq.  mode 1 (CG step): the last
// block turns <p, Ap> into the step alpha (stopping when <p,Ap> <= 0 or
// <r,r> = 0).  mode 2 (ADMM right-hand side): also copy out into pdir and
// reduce <out, out> into scal->rr, marking the CG active.
// ---------------------------------------------------------------------------
// D^T D's two m x m tables as kernel parameters (FP32, m <= 16): they sit in
// the constant bank, and each multiply-add of the unrolled sums takes its
// table entry from there directly, with no shared-memory load per term.
// Other instantiations read shared-memory copies.
template <typename T, int M>
struct LapTab {
    static constexpr bool kParam = sizeof(T) == 4 && M <= 16;
    T G[kParam ? M * M : 1];
    T L[kParam ? M * M : 1];  // lambda2^2 Lt
};

// The last block's update of the solver scalars from the reduced sum of a
// D^T D launch (see the modes above).
__device__ __forceinline__ void lap_scalars(double sum, DevScalars *scal, int mode) {
    if (mode == 1) {
        const double pq = sum, rr = scal->rr;
        scal->pq = pq;
        if (scal->active && pq > 0.0 && rr > 0.0) {
            scal->alpha = rr / pq;
        } else {
            scal->alpha = 0.0;
            scal->active = 0;
        }
    } else if (mode == 2) {
        scal->rr = sum;
        scal->active = 1;
    } else {
        scal->pq = sum;
    }
}

// Resident CTAs per SM asked of the FP32 instantiations: four at m <= 8, two
// (128 registers) at m = 16.
__host__ __device__ constexpr int lap_min_blocks(int M, int T_bytes) {
    return T_bytes == 4 ? (M <= 8 ? 4 : (M == 16 ? 2 : 1)) : 1;
}

template <typename T, int M>
__global__ void __launch_bounds__(kRedThreads, lap_min_blocks(M, sizeof(T)))
    lap_kernel(const T *__restrict__ xv, T *__restrict__ out, T *__restrict__ pdir, const T *PhiF,
               const T *dPhiF, const T *G, const T *Lt, const __grid_constant__ LapTab<T, M> tab, Geo g, T alpha,
               T beta, T lam2sq, double *partials, unsigned *counter, DevScalars *scal, int mode) {
    constexpr bool CT = LapTab<T, M>::kParam;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const T *Gs = sm + 2 * g.nt * M;
    T *Ls = sm + 2 * g.nt * M + M * M;
    if constexpr (!CT) {
        load_tables<T, M>(sm, PhiF, dPhiF, G, Lt, g.nt, true);
        // this block's copy of Lt scaled by lambda2^2 once
        for (int i = threadIdx.x; i < M * M; i += blockDim.x) Ls[i] = lam2sq * Ls[i];
        __syncthreads();
    }
    PartialSum<T> acc;
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    const size_t sy = g.nx, sz = (size_t)g.nx * g.ny;
    // The warps step through the walk together (a lane past the end takes
    // part in the shuffles only): the x neighbours of a voxel are the voxels
    // of the lanes beside it whenever they exist (consecutive steps of the
    // walk are consecutive x of one row), so only the warp's edge lanes read
    // them from memory.
    const int lane = threadIdx.x & 31;
    for (size_t w0 = blockIdx.x * (size_t)blockDim.x + (threadIdx.x & ~31u); w0 < nv;
         w0 += (size_t)gridDim.x * blockDim.x) {
        const size_t it = w0 + lane;
        const bool live = it < nv;
        int x = 0, y = 0, z = 0;
        const size_t v = live ? band_voxel(it, g, x, y, z) : 0;
        T xc[M], ls[M], nb[M];
        if (live) {
            load_coeffs<T, T, M>(xv + v * g.m, g.m, xc);
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) xc[j] = T(0);
        }
#pragma unroll
        for (int j = 0; j < M; ++j) ls[j] = T(0);
        // the six neighbours in the order -x, +x, -y, +y, -z, +z (Neumann: a
        // missing neighbour adds nothing)
        const T *pc = xv + v * g.m;
        auto acc_nb = [&](bool has) {
            if (!has) return;
#pragma unroll
            for (int j = 0; j < M; ++j) ls[j] += xc[j] - nb[j];
        };
        auto add_nb = [&](bool has, long long off) {
            if (!has) return;
            load_coeffs<T, T, M>(pc + off, g.m, nb);
            acc_nb(true);
        };
        if constexpr (M >= 16) {
#pragma unroll
            for (int j = 0; j < M; ++j) nb[j] = __shfl_up_sync(0xffffffffu, xc[j], 1);
            if (lane == 0 && live && x > 0) load_coeffs<T, T, M>(pc - g.m, g.m, nb);
            acc_nb(live && x > 0);
#pragma unroll
            for (int j = 0; j < M; ++j) nb[j] = __shfl_down_sync(0xffffffffu, xc[j], 1);
            if (lane == 31 && live && x + 1 < g.nx) load_coeffs<T, T, M>(pc + g.m, g.m, nb);
            acc_nb(live && x + 1 < g.nx);
        } else {
            add_nb(live && x > 0, -(long long)g.m);
            add_nb(live && x + 1 < g.nx, g.m);
        }
        const long long oy = (long long)sy * g.m, oz = (long long)sz * g.m;
        add_nb(live && y > 0, -oy);
        add_nb(live && y + 1 < g.ny, oy);
        add_nb(live && (z > 0 || g.zlo != 0), -oz);
        add_nb(live && (z + 1 < g.nz || g.zhi != 0), oz);
        if (!live) continue;
        T dotv = T(0);  // this voxel's m products in the compute type (sums in a PartialSum)
        if constexpr (M <= 16) {
            // the row in registers: vector loads and stores of out (and pdir)
            T rv[M], ov[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                T s = T(0);
                if constexpr (CT) {
#pragma unroll
                    for (int j = 0; j < M; ++j) s = fma(tab.G[i * M + j], ls[j], fma(tab.L[i * M + j], xc[j], s));
                } else {
#pragma unroll
                    for (int j = 0; j < M; ++j) s = fma(Gs[i * M + j], ls[j], fma(Ls[i * M + j], xc[j], s));
                }
                rv[i] = alpha * s;
            }
            if (beta != T(0)) {
                load_row<T, M>(out + v * g.m, g.m, ov);
#pragma unroll
                for (int i = 0; i < M; ++i) rv[i] += beta * ov[i];
            }
            store_row<T, M>(out + v * g.m, g.m, rv);
            if (mode == 2) store_row<T, M>(pdir + v * g.m, g.m, rv);
#pragma unroll
            for (int i = 0; i < M; ++i)
                if (i < g.m) dotv = mode == 2 ? fma(rv[i], rv[i], dotv) : fma(xc[i], rv[i], dotv);
        } else {
#pragma unroll 1
            for (int i = 0; i < M; ++i) {
                if (i >= g.m) break;
                T s = T(0);
#pragma unroll
                for (int j = 0; j < M; ++j) s = fma(Gs[i * M + j], ls[j], fma(Ls[i * M + j], xc[j], s));
                const size_t idx = v * g.m + i;
                T r = alpha * s;
                if (beta != T(0)) r += beta * out[idx];
                out[idx] = r;
                if (mode == 2) {
                    pdir[idx] = r;
                    dotv = fma(r, r, dotv);
                } else {
                    dotv = fma(xv[idx], r, dotv);
                }
            }
        }
        acc.add(dotv);
    }
    double vals[1] = {acc.value()}, tot[1];
    if (block_reduce_last<1>(vals, partials, counter, tot)) lap_scalars(tot[0], scal, mode);
}

// ---------------------------------------------------------------------------
// D^T D for FP32 coefficient rows of exactly M = 4, 8 or 16 floats, as a march
// up z over (x, y) tiles.  A CTA of 256 threads owns work items of 32 x 8
// voxels (one voxel per thread) and a run of slices [z0, z1), and walks the
// run up z.  The planes z - 1, z and z + 1 of the tile, with a one-voxel x / y
// halo (34 x 10 voxels of M floats), are in shared memory in a ring of four;
// plane z + 2 is copied by cp.async (16-byte chunks, consecutive threads on
// consecutive chunks of a row) while plane z is computed.  In a staged plane
// the CH = M / 4 chunks of tile voxel k sit in the order c ^ sw(k), with
// sw(k) = (k / (8 / CH)) mod CH, so the rows of any 8 consecutive voxels (a
// quarter warp's 16-byte reads of one neighbour) fall in 8 different bank
// groups: the stencil's seven row reads per voxel are conflict-free
// shared-memory reads instead of strided global loads.  Volumes with few
// tiles are cut into several runs of slices (each run stages its own
// boundary planes) so that the grid still fills the GPU.  The arithmetic per
// voxel is the lap_kernel's (same neighbour order, same sums, tables in the
// constant bank).
// ---------------------------------------------------------------------------
constexpr int kLapTX = 32, kLapTY = 8;
constexpr int kLapHX = kLapTX + 2, kLapHY = kLapTY + 2;
constexpr int kLapPlane = kLapHX * kLapHY;  // voxels of a staged plane
constexpr int kLapRing = 4;                 // planes in the ring
constexpr size_t lap_tile_smem(int M) { return (size_t)kLapRing * kLapPlane * M * sizeof(float); }

// RUNS = false: one run of all nz slices per tile (nruns is 1).
template <int M, bool RUNS>
__global__ void __launch_bounds__(kRedThreads, M == 16 ? 2 : 4)
    lap_tile_kernel(const float *__restrict__ xv, float *__restrict__ out, float *__restrict__ pdir,
                    const __grid_constant__ LapTab<float, M> tab, Geo g, int nruns, float alpha, float beta,
                    double *partials, unsigned *counter, DevScalars *scal, int mode) {
    static_assert(M == 4 || M == 8 || M == 16, "rows of whole 16-byte chunks");
    constexpr int CH = M / 4;  // 16-byte chunks per voxel row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *ring = reinterpret_cast<float4 *>(smem_raw);  // [kLapRing][kLapPlane][CH]
    const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5;
    const int ntx = (g.nx + kLapTX - 1) / kLapTX, nty = (g.ny + kLapTY - 1) / kLapTY;
    if (!RUNS) nruns = 1;
    const int nitems = ntx * nty * nruns;
    // (indices are non-negative: unsigned arithmetic keeps the divisions shifts)
    auto swz = [](int k) { return CH == 1 ? 0 : (int)(((unsigned)k / (8u / CH)) & (CH - 1u)); };
    PartialSum<float> acc;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int tile = RUNS ? item % (ntx * nty) : item, run = RUNS ? item / (ntx * nty) : 0;
        const int x0 = (tile % ntx) * kLapTX, y0 = (tile / ntx) * kLapTY;
        const int z0 = RUNS ? (int)(((long long)run * g.nz) / nruns) : 0;
        const int z1 = RUNS ? (int)(((long long)(run + 1) * g.nz) / nruns) : g.nz;
        const int x = x0 + lx, y = y0 + ly;
        const bool live = x < g.nx && y < g.ny;
        // copy plane zz (z0 - 1 <= zz <= z1 + 1; only planes in memory) into its ring slot
        auto stage = [&](int zz) {
            const bool in_mem = (zz >= 0 && zz < g.nz) || (zz == -1 && g.zlo) || (zz == g.nz && g.zhi);
            if (!in_mem || (RUNS && zz > z1)) return;
            float4 *dst = ring + (size_t)((zz + kLapRing) % kLapRing) * kLapPlane * CH;
            for (int i = tid; i < kLapPlane * CH; i += kRedThreads) {
                const int k = (int)((unsigned)i / CH), c = i - k * CH;
                const int hy = (int)((unsigned)k / kLapHX), hx = k - hy * kLapHX;
                const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
                if (gx < 0 || gx >= g.nx || gy < 0 || gy >= g.ny) continue;
                const float *src = xv + (((long long)zz * g.ny + gy) * g.nx + gx) * M + 4 * c;
                cp_async_16(dst + k * CH + (c ^ swz(k)), src);
            }
        };
        // row of tile voxel k of ring slot sl
        auto row = [&](int sl, int k, float (&r)[M]) {
            const float4 *b = ring + ((size_t)sl * kLapPlane + k) * CH;
            const int sw = swz(k);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const float4 a = b[c ^ sw];
                r[4 * c] = a.x;
                r[4 * c + 1] = a.y;
                r[4 * c + 2] = a.z;
                r[4 * c + 3] = a.w;
            }
        };
        __syncthreads();  // the previous item's reads of the ring are done
        stage(z0 - 1);
        cp_async_commit();
        stage(z0);
        cp_async_commit();
        stage(z0 + 1);
        cp_async_commit();
        for (int z = z0; z < z1; ++z) {
            if (z > z0) __syncthreads();  // every thread is done with step z - 1 (and slot (z + 2) % 4)
            stage(z + 2);
            cp_async_commit();
            cp_async_wait<1>();  // this thread's copies of planes up to z + 1 have landed
            __syncthreads();     // and every thread's
            if (!live) continue;
            const int k = (ly + 1) * kLapHX + lx + 1;
            const int sc = (z + kLapRing) % kLapRing, sb = (z + kLapRing - 1) % kLapRing, sa = (z + 1) % kLapRing;
            float xc[M], ls[M], nb[M];
            row(sc, k, xc);
#pragma unroll
            for (int j = 0; j < M; ++j) ls[j] = 0.0f;
            auto add_nb = [&](bool has, int sl, int kk) {
                if (!has) return;
                row(sl, kk, nb);
#pragma unroll
                for (int j = 0; j < M; ++j) ls[j] += xc[j] - nb[j];
            };
            // the six neighbours in the order -x, +x, -y, +y, -z, +z (as lap_kernel)
            add_nb(x > 0, sc, k - 1);
            add_nb(x + 1 < g.nx, sc, k + 1);
            add_nb(y > 0, sc, k - kLapHX);
            add_nb(y + 1 < g.ny, sc, k + kLapHX);
            add_nb(z > 0 || g.zlo != 0, sb, k);
            add_nb(z + 1 < g.nz || g.zhi != 0, sa, k);
            const size_t v = ((size_t)z * g.ny + y) * g.nx + x;
            float rv[M];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                float s2 = 0.0f;
#pragma unroll
                for (int j = 0; j < M; ++j) s2 = fmaf(tab.G[i * M + j], ls[j], fmaf(tab.L[i * M + j], xc[j], s2));
                rv[i] = alpha * s2;
            }
            // out (and pdir) a 16-byte chunk at a time
            float4 *o4 = reinterpret_cast<float4 *>(out + v * M);
            float dotv = 0.0f;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                float4 r = make_float4(rv[4 * c], rv[4 * c + 1], rv[4 * c + 2], rv[4 * c + 3]);
                if (beta != 0.0f) {
                    const float4 o = o4[c];
                    r.x += beta * o.x;
                    r.y += beta * o.y;
                    r.z += beta * o.z;
                    r.w += beta * o.w;
                }
                o4[c] = r;
                if (mode == 2) reinterpret_cast<float4 *>(pdir + v * M)[c] = r;
                const float rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    dotv = mode == 2 ? fmaf(rr[e], rr[e], dotv) : fmaf(xc[4 * c + e], rr[e], dotv);
            }
            acc.add(dotv);
        }
        cp_async_wait<0>();  // no copy of this item is still in flight
    }
    double vals[1] = {acc.value()}, tot[1];
    if (block_reduce_last<1>(vals, partials, counter, tot)) lap_scalars(tot[0], scal, mode);
}

// ---------------------------------------------------------------------------
// Chambolle-Pock (Fig. 2) step 4: h2 = project(h2 + sigma D ut, lambda1).
// ---------------------------------------------------------------------------
template <typename T, int M, typename F = T>
__global__ void __launch_bounds__(kRedThreads)
    cp_dual_kernel(const T *__restrict__ ut, F *__restrict__ h2, const T *PhiF, const T *dPhiF, Geo g, T sigma,
                   T lambda1, T lambda2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    load_tables<T, M>(sm, PhiF, dPhiF, nullptr, nullptr, g.nt, false);
    const T *dph = sm + g.nt * M;
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < nv; it += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        const size_t v = band_voxel(it, g, x, y, z);
        T uc[M], ex[M], ey[M], ez[M];
        coeff_diffs<T, T, M>(ut, v, x, y, z, g, uc, ex, ey, ez);
        const size_t fb = field_base(v, z, g), fs = frame_stride(g);
        for (int l = 0; l < g.nt; ++l) {
            T d[4];
            grad_frame<T, M>(sm, l, ex, ey, ez, d[0], d[1], d[2]);
            d[3] = dt_frame<T, M>(dph + l * M, lambda2, uc);
            const size_t o = fb + l * fs;
            typename V4<T>::type h = FieldIO<T, F>::ld(h2 + o);
            h.x += sigma * d[0];
            h.y += sigma * d[1];
            h.z += sigma * d[2];
            h.w += sigma * d[3];
            const T n = sqrt(h.x * h.x + h.y * h.y + h.z * h.z + h.w * h.w);
            if (n > lambda1) {
                const T f = lambda1 / n;
                h.x *= f; h.y *= f; h.z *= f; h.w *= f;
            }
            FieldIO<T, F>::st(h2 + o, h);
        }
    }
}

// Fig. 2 steps 5-6: u_new = u - tau (a + D^T h2); ut = u_new + theta (u_new - u).
template <typename T, int M, typename F = T>
__global__ void __launch_bounds__(kRedThreads)
    cp_primal_kernel(T *__restrict__ u, T *__restrict__ ut, const T *__restrict__ a, const F *__restrict__ h2,
                     const T *PhiF, const T *dPhiF, Geo g, T tau, T theta, T lambda2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    load_tables<T, M>(sm, PhiF, dPhiF, nullptr, nullptr, g.nt, false);
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < nv; it += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        const size_t v = band_voxel(it, g, x, y, z);
        T dt[M];
        gradT_voxel<T, M, F>(h2, v, x, y, z, g, sm, lambda2, dt);
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j >= g.m) break;
            const size_t i = v * g.m + j;
            const T uo = u[i];
            const T un = uo - tau * (a[i] + dt[j]);
            u[i] = un;
            ut[i] = un + theta * (un - uo);
        }
    }
}

// sum |D u| (objective TV term) into obj row [1] (row = obj + 3*iter).
template <typename T, int M>
__global__ void __launch_bounds__(kRedThreads)
    tvsum_kernel(const T *__restrict__ u, const T *PhiF, const T *dPhiF, Geo g, T lambda2, double *partials,
                 unsigned *counter, DevScalars *scal, double *obj) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    load_tables<T, M>(sm, PhiF, dPhiF, nullptr, nullptr, g.nt, false);
    const T *dph = sm + g.nt * M;
    PartialSum<T> acc;
    const size_t nv = (size_t)g.nx * g.ny * g.nz;
    for (size_t it = blockIdx.x * (size_t)blockDim.x + threadIdx.x; it < nv; it += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        const size_t v = band_voxel(it, g, x, y, z);
        T uc[M], ex[M], ey[M], ez[M];
        coeff_diffs<T, T, M>(u, v, x, y, z, g, uc, ex, ey, ez);
        for (int l = 0; l < g.nt; ++l) {
            T d[4];
            grad_frame<T, M>(sm, l, ex, ey, ez, d[0], d[1], d[2]);
            d[3] = dt_frame<T, M>(dph + l * M, lambda2, uc);
            acc.add(sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3]));
        }
    }
    double vals[1] = {acc.value()}, tot[1];
    if (block_reduce_last<1>(vals, partials, counter, tot)) obj[3 * (size_t)scal->iter + 1] = tot[0];
}

// ===========================================================================
// Launchers (instantiated per precision in tv_ops_*.cu and tv_calc_*.cu)
// ===========================================================================
// Rows per band of the traversal: one band at one slice holds about
// kBandBytes of u and the dual fields, so the z neighbours (a band apart in
// the walk) stay in L2.  Volumes whose whole slice fits walk slice by slice.
constexpr size_t kBandBytes = 4u << 20;
inline Geo geo(const dr_plan *P) {
    const size_t bpv = (size_t)(4 * P->nt + P->m) * (P->prec == DR_F64 ? 8 : 4);
    const size_t row = std::max<size_t>(1, bpv * (size_t)P->nx);
    const int band = (int)std::max<size_t>(1, std::min<size_t>((size_t)P->ny, kBandBytes / row));
    return Geo{P->nx, P->ny, P->nz, P->m, P->nt, P->z_open_lo, P->z_open_hi, band};
}

template <typename T, int M>
inline size_t tab_smem(const dr_plan *P, bool gl) {
    return sizeof(T) * ((size_t)2 * P->nt * M + (gl ? 2 * M * M : 0));
}

template <typename K>
inline dr_status prep_smem(K kern, size_t smem) {
    return allow_dynamic_smem((const void *)kern, smem);
}

// Blocks of a grid-stride TV launch: as many as the device holds at once, so
// that every block is resident from the start and the walk advances as one
// front (a larger grid leaves the later blocks a second sweep over the
// volume, whose neighbours have long left L2); at most red_grid(n).
// Resident blocks per SM are cached per kernel, dynamic shared memory and
// device.
inline int tv_grid(const void *kern, size_t smem, size_t n) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, size_t, int>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return red_grid(n);
    int per_dev = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(std::make_tuple(kern, smem, dev));
        if (it != cache.end()) per_dev = it->second;
    }
    if (per_dev == 0) {
        int occ = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kRedThreads, smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || occ < 1 || sms < 1) {
            cudaGetLastError();
            return red_grid(n);
        }
        per_dev = occ * sms;
        std::lock_guard<std::mutex> lk(mu);
        cache[std::make_tuple(kern, smem, dev)] = per_dev;
    }
    return std::max(1, std::min(red_grid(n), per_dev));
}

inline dr_status tv_launched(const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DR_OK : cuda_fail(e, what);
}

// TV template sizes: m rounded up to 4, 8, 16 or 32 (tables are padded).
#define DR_TV_MT(...)                                      \
    switch (P->MT) {                                       \
        case 4: { constexpr int M = 4; __VA_ARGS__ }       \
        case 8: { constexpr int M = 8; __VA_ARGS__ }       \
        case 16: { constexpr int M = 16; __VA_ARGS__ }     \
        case 32: { constexpr int M = 32; __VA_ARGS__ }     \
    }                                                      \
    return fail(DR_EINVAL, "tv: unsupported m");

// u = beta u + alpha D^T p with p stored as F; FP32 plans whose frame tables
// fit the kernel parameter take them from the constant bank.
template <typename T, typename S, int M, typename F>
inline dr_status launch_gradT(dr_plan *P, const F *p, S *u_s, T *u_c, double lambda2, double alpha, double beta,
                              cudaStream_t st, const char *what) {
    FrameTab<T> ft{};
    const bool ct = sizeof(T) == 4 && P->nt * M <= kFrameTabMax;
    if (ct)
        for (int i = 0; i < P->nt * M; ++i) {
            ft.ph[i] = (T)P->h_phif[i];
            ft.dph[i] = (T)P->h_dphif[i];
        }
    auto kern = ct ? gradT_kernel<T, S, M, F, true> : gradT_kernel<T, S, M, F, false>;
    const size_t smem = ct ? 0 : tab_smem<T, M>(P, false);
    dr_status s = prep_smem(kern, smem);
    if (s != DR_OK) return s;
    const int grid = tv_grid((const void *)kern, smem, nvox(P));
    kern<<<grid, kRedThreads, smem, st>>>(p, u_s, u_c, (const T *)P->d_PhiF, (const T *)P->d_dPhiF, geo(P), (T)lambda2,
                                          (T)alpha, (T)beta, ft);
    return tv_launched(what);
}

// Kernels whose coefficient input may be stored in S (bf16 for BF16 plans).
template <typename T, typename S>
struct TvOps {
    static dr_status grad(dr_plan *P, const void *u, void *p, double lambda2, cudaStream_t st) {
        DR_TV_MT({
            auto kern = grad_kernel<T, S, M>;
            const size_t smem = tab_smem<T, M>(P, false);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>((const S *)u, (T *)p, (const T *)P->d_PhiF,
                                                   (const T *)P->d_dPhiF, geo(P), (T)lambda2);
            return tv_launched("grad_kernel");
        })
    }
    static dr_status grad_adj(dr_plan *P, const void *p, void *u, bool calc, double lambda2, double alpha,
                              double beta, cudaStream_t st) {
        DR_TV_MT({
            return launch_gradT<T, S, M, T>(P, (const T *)p, calc ? nullptr : (S *)u, calc ? (T *)u : nullptr,
                                            lambda2, alpha, beta, st, "gradT_kernel");
        })
    }
    static dr_status prox(dr_plan *P, const void *u, void *mu, void *w, double rho, double lambda1, double lambda2,
                          double *obj_row, cudaStream_t st) {
        DR_TV_MT({
            auto kern = prox_kernel<T, S, M>;
            const size_t smem = tab_smem<T, M>(P, false);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>(
                (const S *)u, (T *)mu, (T *)w, (const T *)P->d_PhiF, (const T *)P->d_dPhiF, geo(P), (T)rho,
                (T)lambda1, (T)lambda2, P->d_partials + kSlotProx * kRedSlotStride, P->d_counters + kSlotProx,
                P->d_scal, obj_row, obj_row ? 1 : 0);
            return tv_launched("prox_kernel");
        })
    }
};

// Kernels on compute-typed solver vectors only.
template <typename T>
struct TvCalc {
    static dr_status lap(dr_plan *P, const void *x, void *out, void *pdir, double alpha, double beta,
                         double lambda2, int mode, cudaStream_t st) {
        DR_TV_MT({
            auto kern = lap_kernel<T, M>;
            LapTab<T, M> tab{};
            if constexpr (LapTab<T, M>::kParam) {
                const double l2 = lambda2 * lambda2;
                for (int k = 0; k < M * M; ++k) {
                    tab.G[k] = (T)P->h_G[k];
                    tab.L[k] = (T)(l2 * P->h_Lt[k]);
                }
            }
            const int slot = mode == 2 ? kSlotRhs : kSlotLap;
            if constexpr (sizeof(T) == 4 && (M == 4 || M == 8 || M == 16)) {
                // rows of exactly M floats, 16-byte aligned, at least one full tile width:
                // the z-marching form with the rows staged in shared memory
                auto al16 = [](const void *q) { return ((uintptr_t)q & 15u) == 0; };
                if (P->m == M && P->nx >= kLapTX && al16(x) && al16(out) && (mode != 2 || al16(pdir))) {
                    const size_t tsm = lap_tile_smem(M);
                    dr_status s2 = prep_smem(lap_tile_kernel<M, true>, tsm);
                    if (s2 == DR_OK) s2 = prep_smem(lap_tile_kernel<M, false>, tsm);
                    if (s2 != DR_OK) return s2;
                    const Geo gg = geo(P);
                    const int ntiles = ((gg.nx + kLapTX - 1) / kLapTX) * ((gg.ny + kLapTY - 1) / kLapTY);
                    const int resident = tv_grid((const void *)lap_tile_kernel<M, false>, tsm, nvox(P));
                    // runs of slices per tile: enough work items for two per resident CTA
                    const int nruns = std::max(1, std::min(gg.nz, (2 * resident + ntiles - 1) / ntiles));
                    auto tk = nruns > 1 ? lap_tile_kernel<M, true> : lap_tile_kernel<M, false>;
                    const int grid = std::max(1, std::min(ntiles * nruns, resident));
                    tk<<<grid, kRedThreads, tsm, st>>>((const float *)x, (float *)out, (float *)pdir, tab, gg, nruns,
                                                       (float)alpha, (float)beta, P->d_partials + slot * kRedSlotStride,
                                                       P->d_counters + slot, P->d_scal, mode);
                    return tv_launched("lap_tile_kernel");
                }
            }
            const size_t smem = LapTab<T, M>::kParam ? 0 : tab_smem<T, M>(P, true);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>(
                (const T *)x, (T *)out, (T *)pdir, (const T *)P->d_PhiF, (const T *)P->d_dPhiF, (const T *)P->d_G,
                (const T *)P->d_Lt, tab, geo(P), (T)alpha, (T)beta, (T)(lambda2 * lambda2),
                P->d_partials + slot * kRedSlotStride, P->d_counters + slot, P->d_scal, mode);
            return tv_launched("lap_kernel");
        })
    }
    static dr_status cp_dual(dr_plan *P, const void *ut, void *h2, double sigma, double lambda1, double lambda2,
                             cudaStream_t st) {
        DR_TV_MT({
            auto kern = cp_dual_kernel<T, M>;
            const size_t smem = tab_smem<T, M>(P, false);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>((const T *)ut, (T *)h2, (const T *)P->d_PhiF,
                                                   (const T *)P->d_dPhiF, geo(P), (T)sigma,
                                                   (T)lambda1, (T)lambda2);
            return tv_launched("cp_dual_kernel");
        })
    }
    static dr_status cp_primal(dr_plan *P, void *u, void *ut, const void *a, const void *h2, double tau,
                               double theta, double lambda2, cudaStream_t st) {
        DR_TV_MT({
            auto kern = cp_primal_kernel<T, M>;
            const size_t smem = tab_smem<T, M>(P, false);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>((T *)u, (T *)ut, (const T *)a, (const T *)h2,
                                                   (const T *)P->d_PhiF, (const T *)P->d_dPhiF,
                                                   geo(P), (T)tau, (T)theta, (T)lambda2);
            return tv_launched("cp_primal_kernel");
        })
    }
    static dr_status tv_sum(dr_plan *P, const void *u, double lambda2, double *obj, cudaStream_t st) {
        DR_TV_MT({
            auto kern = tvsum_kernel<T, M>;
            const size_t smem = tab_smem<T, M>(P, false);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>((const T *)u, (const T *)P->d_PhiF,
                                                   (const T *)P->d_dPhiF, geo(P), (T)lambda2,
                                                   P->d_partials + kSlotTv * kRedSlotStride,
                                                   P->d_counters + kSlotTv, P->d_scal, obj);
            return tv_launched("tvsum_kernel");
        })
    }
};

// The solver's kernels on dual fields stored in bf16 (compute-typed float
// coefficient vectors; FP32 arithmetic).
struct TvFieldsBF16 {
    static dr_status grad_adj(dr_plan *P, const void *p, void *u, double lambda2, double alpha, double beta,
                              cudaStream_t st) {
        typedef float T;
        DR_TV_MT({
            return launch_gradT<T, T, M, bf16>(P, (const bf16 *)p, nullptr, (T *)u, lambda2, alpha, beta, st,
                                               "gradT_kernel (bf16 field)");
        })
    }
    static dr_status prox(dr_plan *P, const void *u, void *mu, void *w, double rho, double lambda1, double lambda2,
                          double *obj_row, cudaStream_t st) {
        typedef float T;
        DR_TV_MT({
            auto kern = prox_kernel<T, T, M, bf16>;
            const size_t smem = tab_smem<T, M>(P, false);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>(
                (const T *)u, (bf16 *)mu, (bf16 *)w, (const T *)P->d_PhiF, (const T *)P->d_dPhiF, geo(P), (T)rho,
                (T)lambda1, (T)lambda2, P->d_partials + kSlotProx * kRedSlotStride, P->d_counters + kSlotProx,
                P->d_scal, obj_row, obj_row ? 1 : 0);
            return tv_launched("prox_kernel (bf16 fields)");
        })
    }
    static dr_status cp_dual(dr_plan *P, const void *ut, void *h2, double sigma, double lambda1, double lambda2,
                             cudaStream_t st) {
        typedef float T;
        DR_TV_MT({
            auto kern = cp_dual_kernel<T, M, bf16>;
            const size_t smem = tab_smem<T, M>(P, false);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>((const T *)ut, (bf16 *)h2, (const T *)P->d_PhiF,
                                                   (const T *)P->d_dPhiF, geo(P), (T)sigma,
                                                   (T)lambda1, (T)lambda2);
            return tv_launched("cp_dual_kernel (bf16 field)");
        })
    }
    static dr_status cp_primal(dr_plan *P, void *u, void *ut, const void *a, const void *h2, double tau,
                               double theta, double lambda2, cudaStream_t st) {
        typedef float T;
        DR_TV_MT({
            auto kern = cp_primal_kernel<T, M, bf16>;
            const size_t smem = tab_smem<T, M>(P, false);
            dr_status s = prep_smem(kern, smem);
            if (s != DR_OK) return s;
            const int grid = tv_grid((const void *)kern, smem, nvox(P));
            kern<<<grid, kRedThreads, smem, st>>>((T *)u, (T *)ut, (const T *)a, (const bf16 *)h2,
                                                   (const T *)P->d_PhiF, (const T *)P->d_dPhiF,
                                                   geo(P), (T)tau, (T)theta, (T)lambda2);
            return tv_launched("cp_primal_kernel (bf16 field)");
        })
    }
};

extern template struct TvOps<float, float>;
extern template struct TvOps<float, bf16>;
extern template struct TvOps<double, double>;
extern template struct TvCalc<float>;
extern template struct TvCalc<double>;

}  // namespace dr
