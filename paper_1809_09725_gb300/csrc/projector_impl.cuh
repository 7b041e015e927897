// projector_impl.cuh -- dynamic parallel-beam projector pair of the time-domain
// decomposition (Sec. 4, Eqs. radapr and radadjapr):
//
//   forward  g[z][k][b] = sum_j phi_j(t_k) (R_{theta_k} u_j[z])(s_b)
//   adjoint  u_j[z]    += sum_k phi_j(t_k) (R*_{theta_k} g[z][k])
//
// R is the Joseph ray-driven projector and R* its exact transpose, written
// pixel-driven.  Both kernels are FP32 FMA bound on GB300, not HBM bound.
//
// Forward (fwd_kernel): one CTA per (slice, block of P projections that step
// along the same image axis).  The CTA walks the image in strips of R lines;
// for each strip it first synthesises the P object states
//     f(x, t_k) = sum_j phi_j(t_k) u_j(x)
// into shared memory (the basis combine, m FMAs per pixel and projection,
// u read once per P projections), then every thread advances its rays
// through the strip with a 32.32 fixed-point sample position (exact to 2^-32
// per step, no float rounding of large coordinates, no float->int
// conversion) and two scalar shared-memory taps per sample.
//
// Adjoint (adj_kernel): one CTA per (slice, 8*VPT x 16 voxel tile), 128
// threads, VPT voxels per thread, all m accumulators per voxel in registers.
// Projections are consumed in stages of 32; for each stage one warp computes
// where the tile's footprint falls on each detector row and issues one TMA
// tile load per projection (a window of Wb bins, zero filled outside the
// detector) plus one TMA load of the 32 basis rows phi_j(t_k), completing on
// an mbarrier; three stages are in flight.  Per (voxel, projection) the
// kernel forms the two-bin triangle footprint of half-width c = max(|cos|,
// |sin|) and does m FMAs into the accumulators.
#include <algorithm>
#include <cmath>

#pragma once
#include "dr_device.cuh"

namespace dr {

// ===========================================================================
// Forward
// ===========================================================================
__host__ __device__ inline size_t fwd_align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <typename S, typename T, int M>
__global__ void __launch_bounds__(kFwdThreads, (sizeof(T) == 4 && M <= 8) ? 3 : 1)
    fwd_kernel(const S *__restrict__ u, S *__restrict__ out, const S *__restrict__ gm,
               const FwdProj *__restrict__ proj, const T *__restrict__ phip, const int *__restrict__ blocks,
               int nx, int ny, int ns, int K, int m, int MP, int P, int R, int mode, T sigma) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    size_t off = 0;
    T *phi_s = reinterpret_cast<T *>(smem_raw + off);             // [P][M]
    off += fwd_align16((size_t)P * M * sizeof(T));
    T *scale_s = reinterpret_cast<T *>(smem_raw + off);           // [P]
    off += fwd_align16((size_t)P * sizeof(T));
    long long *bfx_s = reinterpret_cast<long long *>(smem_raw + off);  // [P] (fixed point)
    off += fwd_align16((size_t)P * sizeof(long long));
    T *bd_s = reinterpret_cast<T *>(smem_raw + off);              // [P] (B as T, FP64 path)
    off += fwd_align16((size_t)P * sizeof(T));
    T *frames = reinterpret_cast<T *>(smem_raw + off);            // [P][R][wpad]

    const int tid = threadIdx.x;
    const int z = blockIdx.y;
    const int *blk = blocks + (size_t)blockIdx.x * P;
    const int branch = proj[blk[0]].branch;
    const int W = branch ? ny : nx;  // samples along a line
    const int H = branch ? nx : ny;  // lines
    const int wpad = W + 2 * kFwdGuard + 1;

    for (int i = tid; i < P * M; i += kFwdThreads) {
        const int p = i / M, j = i - p * M;
        const int k = blk[p];
        phi_s[i] = (k >= 0 && j < m) ? phip[(size_t)k * MP + j] : T(0);
    }
    for (int p = tid; p < P; p += kFwdThreads) {
        const int k = blk[p];
        const FwdProj f = proj[k >= 0 ? k : blk[0]];
        if constexpr (sizeof(T) == 8) scale_s[p] = (T)f.scale_d;
        else scale_s[p] = (T)f.scale;
        bfx_s[p] = f.B_fx;
        bd_s[p] = (T)f.B;
    }
    for (int i = tid; i < P * R * wpad; i += kFwdThreads) frames[i] = T(0);

    // ray state: ray id = tid + q * threads, (p, b) = (id / ns, id % ns)
    const int nrays = P * ns;
    long long x0fx[kFwdRPT];
    T x0d[kFwdRPT];
    int lo[kFwdRPT], hi[kFwdRPT];
    T acc[kFwdRPT];
#pragma unroll
    for (int q = 0; q < kFwdRPT; ++q) {
        const int rid = tid + q * kFwdThreads;
        acc[q] = T(0);
        lo[q] = 1;
        hi[q] = 0;
        x0fx[q] = 0;
        x0d[q] = T(0);
        if (rid < nrays) {
            const int p = rid / ns, b = rid - p * ns;
            const int k = blk[p];
            if (k >= 0) {
                const FwdProj f = proj[k];
                x0fx[q] = f.C_fx + (long long)b * f.A_fx;
                if constexpr (sizeof(T) == 8) x0d[q] = f.C + (double)b * f.A;
                // rows whose sample can fall inside (-1, W); estimated in float
                // with a one-row margin (the tap index is clamped anyway)
                const float xf = f.Cf + (float)b * f.Af;
                const float Bf = f.Bf;
                if (fabsf(Bf) < 1e-2f) {
                    lo[q] = 0;
                    hi[q] = H - 1;
                } else {
                    const float r1 = (-1.0f - xf) / Bf, r2 = ((float)W - xf) / Bf;
                    float rmin = fminf(r1, r2), rmax = fmaxf(r1, r2);
                    rmin = fmaxf(rmin, -4.0f);
                    rmax = fminf(rmax, (float)H + 4.0f);
                    lo[q] = max(0, (int)floorf(rmin) - 1);
                    hi[q] = min(H - 1, (int)ceilf(rmax) + 1);
                }
            }
        }
    }
    __syncthreads();

    const size_t zoff = (size_t)z * ny * nx;
    for (int r0 = 0; r0 < H; r0 += R) {
        const int nl = min(R, H - r0);
        // ---- synthesis of the P object states on lines [r0, r0+nl) ----
        // A thread synthesises two pixels (qq and qq + kFwdThreads) per pass,
        // so every phi row read from shared memory (as 16-byte vectors when
        // they are float rows) serves both; each f is the same FMA chain
        // over j as for one pixel.
        const int npx = nl * W;
        auto pixel_of = [&](int qq, int &rl, int &a) -> size_t {
            if (branch == 0) {
                rl = qq / W;
                a = qq - rl * W;
                return zoff + (size_t)(r0 + rl) * nx + a;
            }
            a = qq / nl;
            rl = qq - a * nl;
            return zoff + (size_t)a * nx + (r0 + rl);
        };
        for (int qq = tid; qq < npx; qq += 2 * kFwdThreads) {
            const bool two = qq + kFwdThreads < npx;
            int rlA, aA, rlB = 0, aB = 0;
            const size_t pixA = pixel_of(qq, rlA, aA);
            const size_t pixB = two ? pixel_of(qq + kFwdThreads, rlB, aB) : pixA;
            T uA[M], uB[M];
            load_coeffs<T, S, M>(u + pixA * m, m, uA);
            load_coeffs<T, S, M>(u + pixB * m, m, uB);
            T *dstA = frames + (size_t)rlA * wpad + kFwdGuard + aA;
            T *dstB = frames + (size_t)rlB * wpad + kFwdGuard + aB;
            for (int p = 0; p < P; ++p) {
                T ph[M];
                if constexpr (sizeof(T) == 4 && (M % 4) == 0) {
#pragma unroll
                    for (int c = 0; c < M / 4; ++c) {
                        const float4 v4 = reinterpret_cast<const float4 *>(phi_s + p * M)[c];
                        ph[4 * c] = v4.x;
                        ph[4 * c + 1] = v4.y;
                        ph[4 * c + 2] = v4.z;
                        ph[4 * c + 3] = v4.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < M; ++j) ph[j] = phi_s[p * M + j];
                }
                T fA = T(0), fB = T(0);
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    fA = fma(ph[j], uA[j], fA);
                    fB = fma(ph[j], uB[j], fB);
                }
                dstA[(size_t)p * R * wpad] = fA;
                if (two) dstB[(size_t)p * R * wpad] = fB;
            }
        }
        __syncthreads();
        // ---- march rays through the strip ----
#pragma unroll
        for (int q = 0; q < kFwdRPT; ++q) {
            const int rs = max(lo[q], r0), re = min(hi[q], r0 + nl - 1);
            if (rs > re) continue;
            const int p = (tid + q * kFwdThreads) / ns;
            const T *row = frames + ((size_t)p * R + (rs - r0)) * wpad + kFwdGuard;
            T a = acc[q];
            if constexpr (sizeof(T) == 4) {
                const long long bfx = bfx_s[p];
                long long x = x0fx[q] + (long long)rs * bfx;
                for (int r = rs; r <= re; ++r) {
                    int i0 = (int)(x >> 32);
                    i0 = min(max(i0, -2), W);
                    const float w = __uint_as_float(0x3F800000u | ((unsigned)x >> 9)) - 1.0f;
                    const float f0 = row[i0], f1 = row[i0 + 1];
                    a += fmaf(w, f1 - f0, f0);
                    x += bfx;
                    row += wpad;
                }
            } else {
                const T bd = bd_s[p];
                for (int r = rs; r <= re; ++r) {
                    const T xi = x0d[q] + (T)r * bd;
                    const T fl = floor(xi);
                    const T w = xi - fl;
                    int i0 = (int)fl;
                    i0 = min(max(i0, -2), W);
                    const T f0 = row[i0], f1 = row[i0 + 1];
                    a += (T(1) - w) * f0 + w * f1;
                    row += wpad;
                }
            }
            acc[q] = a;
        }
        __syncthreads();
    }

    // ---- epilogue ----
#pragma unroll
    for (int q = 0; q < kFwdRPT; ++q) {
        const int rid = tid + q * kFwdThreads;
        if (rid >= nrays) continue;
        const int p = rid / ns, b = rid - p * ns;
        const int k = blk[p];
        if (k < 0) continue;
        const size_t idx = ((size_t)z * K + k) * ns + b;
        const T val = acc[q] * scale_s[p];
        if (mode == 0) {
            stc<T>(out + idx, val);
        } else if (mode == 1) {
            stc<T>(out + idx, val - ldc<T>(gm + idx));
        } else {
            const T h = ldc<T>(out + idx);
            stc<T>(out + idx, (h + sigma * val - sigma * ldc<T>(gm + idx)) / (T(1) + sigma));
        }
    }
}

template <typename S, typename T, int M>
inline dr_status fwd_launch_t(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                              cudaStream_t st) {
    const int Pp = P->fwd_P, R = P->fwd_R;
    const int Wmax = std::max(P->nx, P->ny);
    const int wpad = Wmax + 2 * kFwdGuard + 1;
    const size_t head = fwd_align16((size_t)Pp * M * sizeof(T)) + 2 * fwd_align16((size_t)Pp * sizeof(T)) +
                        fwd_align16((size_t)Pp * sizeof(long long));
    const size_t smem = head + sizeof(T) * (size_t)Pp * R * wpad;
    auto kern = fwd_kernel<S, T, M>;
    {
        dr_status s = allow_dynamic_smem((const void *)kern, smem);
        if (s != DR_OK) return s;
    }
    dim3 grid(P->n_fwd_blocks, P->nz);
    kern<<<grid, kFwdThreads, smem, st>>>((const S *)u, (S *)out, (const S *)gm, P->d_fwd, (const T *)P->d_PhiP,
                                          P->d_fwd_blocks, P->nx, P->ny, P->ns, P->K, P->m, P->MP, Pp, R, mode,
                                          (T)sigma);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fwd_kernel launch");
    return DR_OK;
}

// ===========================================================================
// Adjoint
// ===========================================================================
template <typename T>
struct AdjPrm;
template <>
struct alignas(16) AdjPrm<float> {
    float c, s, c8, qb;      // cos, sin, 8*cos, (window-relative origin position) - 1/2
    float e0, inv_c2;       // 1/c - 1/(2c^2), 1/c^2
    int idx_base, pad_;     // integer part of the origin position minus the float magic
};
template <>
struct alignas(16) AdjPrm<double> {
    double c, s, c8, qb;    // qb: fractional origin position (no shift)
    double inv_c, inv_c2;
    int idx_base, pad_[3];
};

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: adding it rounds to an integer
constexpr int kMagicInt = 0x4B400000;

template <int M>
struct AdjShape {
    static constexpr int VPT = (M <= 8) ? 4 : ((M <= 16) ? 2 : 1);
    static constexpr int TX = 8 * VPT;
};

// Window geometry shared by host and device.
__host__ __device__ inline int adj_align(int s_bytes) { return 16 / s_bytes; }

template <typename S, typename T, int M>
__global__ void __launch_bounds__(kAdjThreads)
    adj_kernel(const __grid_constant__ CUtensorMap tm_g, const __grid_constant__ CUtensorMap tm_phi,
               const S *__restrict__ g, const T *__restrict__ phip, const AdjProj *__restrict__ proj,
               S *__restrict__ u_s, T *__restrict__ u_c, int nx, int ny, int ns, int K, int m, int MP, int Wb,
               int wbs, int use_tma, T alpha, T beta, int *status) {
    constexpr int VPT = AdjShape<M>::VPT;
    constexpr int TX = AdjShape<M>::TX;
    constexpr int TY = kAdjTY;
    constexpr int PP = kAdjP;
    constexpr int NST = kAdjStages;
    constexpr int ALIGN = 16 / (int)sizeof(S);

    extern __shared__ __align__(128) unsigned char adj_smem_raw[];
    // the launch adds 128 bytes so the base can be rounded up to 128 B (TMA destination alignment)
    // round up to 128 B by pointer arithmetic on the __shared__ array, so the
    // compiler keeps addressing it as shared memory (LDS, not generic loads)
    unsigned char *smem_raw = adj_smem_raw + ((128u - (smem_u32(adj_smem_raw) & 127u)) & 127u);
    // per stage: window [PP][wbs] S (rows 128-B aligned), phi [PP][MP] T, prm [PP]
    const size_t win_bytes = (size_t)PP * wbs * sizeof(S);
    const size_t phi_bytes = (((size_t)PP * MP * sizeof(T)) + 127) & ~(size_t)127;
    const size_t prm_bytes = (((size_t)PP * sizeof(AdjPrm<T>)) + 127) & ~(size_t)127;
    const size_t stage_bytes = win_bytes + phi_bytes + prm_bytes;
    __shared__ __align__(8) uint64_t full[NST];
    auto win_s = [&](int st) { return reinterpret_cast<S *>(smem_raw + st * stage_bytes); };
    auto phi_s = [&](int st) { return reinterpret_cast<T *>(smem_raw + st * stage_bytes + win_bytes); };
    auto prm_s = [&](int st) {
        return reinterpret_cast<AdjPrm<T> *>(smem_raw + st * stage_bytes + win_bytes + phi_bytes);
    };

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntx = (nx + TX - 1) / TX;
    const int x0 = (blockIdx.x % ntx) * TX, y0 = (blockIdx.x / ntx) * TY;
    const int z = blockIdx.y;
    const int xo = x0 + TX / 2, yo = y0 + TY / 2;  // tile origin voxel
    const int tx = tid & 7, ty = tid >> 3;
    const int dx0 = x0 + tx - xo, dy = y0 + ty - yo;
    const int nkb = (K + PP - 1) / PP;

    // Compute one projection's window and parameters (one lane per projection).
    auto stage_params = [&](int st, int kb, int p, int &wb0_out, int &krow) {
        const int k = kb * PP + p;
        const int kk = k < K ? k : K - 1;
        const AdjProj a = proj[kk];
        const double posO = xo * a.c + yo * a.s + a.C0;
        const double dxa = (double)(-TX / 2), dxb = (double)(TX / 2 - 1);
        const double dya = (double)(-TY / 2), dyb = (double)(TY / 2 - 1);
        const double emin = posO + fmin(dxa * a.c, dxb * a.c) + fmin(dya * a.s, dyb * a.s);
        int wb0 = (int)floor(emin) - 1;
        wb0 = (wb0 >= 0) ? (wb0 / ALIGN) * ALIGN : -(((-wb0) + ALIGN - 1) / ALIGN) * ALIGN;
        const double rel = posO - wb0;
        const double ri = floor(rel);
        AdjPrm<T> pr;
        if constexpr (sizeof(T) == 4) {
            const float inv_c = (float)a.inv_c;
            pr.c = (float)a.c;
            pr.s = (float)a.s;
            pr.c8 = (float)(8.0 * a.c);
            pr.qb = (float)(rel - ri) - 0.5f;
            pr.inv_c2 = (float)(a.inv_c * a.inv_c);
            pr.e0 = (float)(a.inv_c - 0.5 * a.inv_c * a.inv_c);
            (void)inv_c;
            pr.idx_base = (int)ri - kMagicInt;
            pr.pad_ = 0;
        } else {
            pr.c = a.c;
            pr.s = a.s;
            pr.c8 = 8.0 * a.c;
            pr.qb = rel - ri;
            pr.inv_c = a.inv_c;
            pr.inv_c2 = a.inv_c * a.inv_c;
            pr.idx_base = (int)ri;
        }
        prm_s(st)[p] = pr;
        wb0_out = wb0;
        krow = z * K + kk;
    };

    // TMA producer: warp 0 fills stage st with projection block kb.
    auto issue = [&](int st, int kb) {
        int wb0 = 0, krow = 0;
        if (lane < PP) stage_params(st, kb, lane, wb0, krow);
        __syncwarp();
        if (lane == 0)
            mbar_arrive_expect_tx(&full[st], (unsigned)(PP * Wb * sizeof(S) + PP * MP * sizeof(T)));
        __syncwarp();
        if (lane < PP) tma_load_2d(win_s(st) + (size_t)lane * wbs, &tm_g, wb0, krow, &full[st]);
        if (lane == 0) tma_load_2d(phi_s(st), &tm_phi, 0, kb * PP, &full[st]);
        if (lane != 0) mbar_arrive(&full[st]);
    };

    // Plain-load staging (unaligned rows): all threads, synchronous.
    __shared__ int wb0_s[PP];
    auto fill_plain = [&](int kb) {
        if (warp == 0) {
            int wb0 = 0, krow = 0;
            if (lane < PP) {
                stage_params(0, kb, lane, wb0, krow);
                wb0_s[lane] = wb0;
            }
        }
        __syncthreads();
        S *win = win_s(0);
        for (int i = tid; i < PP * Wb; i += kAdjThreads) {
            const int p = i / Wb, c = i - p * Wb;
            const int k = kb * PP + p;
            const int b = wb0_s[p] + c;
            S v = S(0.0f);
            if (k < K && b >= 0 && b < ns) v = g[((size_t)z * K + k) * ns + b];
            win[(size_t)p * wbs + c] = v;
        }
        T *ph = phi_s(0);
        for (int i = tid; i < PP * MP; i += kAdjThreads) {
            const int p = i / MP, j = i - p * MP;
            const int k = kb * PP + p;
            ph[i] = (k < K) ? phip[(size_t)k * MP + j] : T(0);
        }
        __syncthreads();
    };

    if (use_tma) {
        if (tid == 0) {
            for (int s = 0; s < NST; ++s) mbar_init(&full[s], 32);
            fence_mbar_init();
        }
        __syncthreads();
        if (warp == 0)
            for (int s = 0; s < NST && s < nkb; ++s) issue(s, s);
    }

    T acc[VPT][M];
#pragma unroll
    for (int v = 0; v < VPT; ++v)
#pragma unroll
        for (int j = 0; j < M; ++j) acc[v][j] = T(0);

    const T dxf = (T)dx0, dyf = (T)dy;
    for (int kb = 0; kb < nkb; ++kb) {
        const int st = use_tma ? (kb % NST) : 0;
        bool bad = false;
        if (use_tma) bad = !mbar_wait_bounded(&full[st], (unsigned)((kb / NST) & 1), status, 2000000000ull);
        else fill_plain(kb);
        if (!bad) {
            const S *win = win_s(st);
            const T *phs = phi_s(st);
            const AdjPrm<T> *prm = prm_s(st);
            const int np = min(PP, K - kb * PP);
            for (int p = 0; p < np; ++p) {
                const AdjPrm<T> a = prm[p];
                T ph[M];
                if constexpr (sizeof(T) == 4 && (M % 4) == 0) {
                    // phi rows are MP = M rounded up to 4 floats, 16-byte aligned
#pragma unroll
                    for (int c = 0; c < M / 4; ++c) {
                        const float4 v4 = reinterpret_cast<const float4 *>(phs + p * MP)[c];
                        ph[4 * c] = v4.x;
                        ph[4 * c + 1] = v4.y;
                        ph[4 * c + 2] = v4.z;
                        ph[4 * c + 3] = v4.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < M; ++j) ph[j] = phs[p * MP + j];
                }
                const S *w = win + (size_t)p * wbs;
                if constexpr (sizeof(T) == 4) {
                    float q = fmaf(dyf, a.s, fmaf(dxf, a.c, a.qb));
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const float t = q + kMagic;
                        const float fl = t - kMagic;
                        const float d = q - fl;
                        const int idx = __float_as_int(t) + a.idx_base;
                        const float w0 = fmaxf(0.0f, fmaf(-d, a.inv_c2, a.e0));
                        const float w1 = fmaxf(0.0f, fmaf(d, a.inv_c2, a.e0));
                        const float val = fmaf(w1, ldc<float>(w + idx + 1), w0 * ldc<float>(w + idx));
#pragma unroll
                        for (int j = 0; j < M; ++j) acc[v][j] = fmaf(ph[j], val, acc[v][j]);
                        q += a.c8;
                    }
                } else {
                    T q = a.qb + dxf * a.c + dyf * a.s;
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const T fl = floor(q);
                        const T d0 = q - fl;
                        const int idx = (int)fl + a.idx_base;
                        const T w0 = fmax(T(0), a.inv_c - d0 * a.inv_c2);
                        const T w1 = fmax(T(0), a.inv_c - (T(1) - d0) * a.inv_c2);
                        const T val = w0 * ldc<T>(w + idx) + w1 * ldc<T>(w + idx + 1);
#pragma unroll
                        for (int j = 0; j < M; ++j) acc[v][j] += ph[j] * val;
                        q += a.c8;
                    }
                }
            }
        }
        if (use_tma) {
            if (__syncthreads_or(bad)) {
                // give up: let loads already in flight land (bounded), then leave
                if (tid == 0)
                    for (int s = kb; s < nkb && s < kb + NST; ++s)
                        mbar_wait_bounded(&full[s % NST], (unsigned)((s / NST) & 1), status, 100000000ull);
                return;
            }
            if (warp == 0 && kb + NST < nkb) issue(st, kb + NST);
        } else {
            __syncthreads();
        }
    }

    // ---- epilogue: u = alpha * acc + beta * u ----
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int x = x0 + tx + 8 * v, y = y0 + ty;
        if (x >= nx || y >= ny) continue;
        const size_t base = (((size_t)z * ny + y) * nx + x) * m;
        if (u_c) {
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (j < m) {
                    T r = alpha * acc[v][j];
                    if (beta != T(0)) r += beta * u_c[base + j];
                    u_c[base + j] = r;
                }
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (j < m) {
                    T r = alpha * acc[v][j];
                    if (beta != T(0)) r += beta * ldc<T>(u_s + base + j);
                    stc<T>(u_s + base + j, r);
                }
        }
    }
}

template <typename S, typename T, int M>
inline dr_status adj_launch_t(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                              cudaStream_t st) {
    constexpr int TX = AdjShape<M>::TX;
    const int ALIGN = 16 / (int)sizeof(S);
    const double ext = std::sqrt((double)(TX - 1) * (TX - 1) + (double)(kAdjTY - 1) * (kAdjTY - 1));
    int Wb = (int)std::ceil(ext) + 5 + ALIGN;
    Wb = (Wb + ALIGN - 1) / ALIGN * ALIGN;
    const int row_bytes = (int)((Wb * sizeof(S) + 127) / 128 * 128);
    const int wbs = row_bytes / (int)sizeof(S);
    const size_t win_bytes = (size_t)kAdjP * wbs * sizeof(S);
    const size_t phi_bytes = (((size_t)kAdjP * P->MP * sizeof(T)) + 127) & ~(size_t)127;
    const size_t prm_bytes = (((size_t)kAdjP * sizeof(AdjPrm<T>)) + 127) & ~(size_t)127;
    const size_t smem = (win_bytes + phi_bytes + prm_bytes) * kAdjStages + 128;

    // TMA needs 16-byte aligned rows and base addresses.
    const bool aligned = ((size_t)P->ns * sizeof(S)) % 16 == 0 && ((uintptr_t)g % 16) == 0 &&
                         ((uintptr_t)P->d_PhiP % 16) == 0;
    CUtensorMap tm_g{}, tm_phi{};
    int use_tma = 0;
    if (aligned) {
        const CUtensorMapDataType dt = sizeof(S) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                       : sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                        : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        const CUtensorMapDataType dtp = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
        const bool ok1 = encode_tensor_map_2d(&tm_g, dt, const_cast<void *>(g), (uint64_t)P->ns,
                                              (uint64_t)P->nz * P->K, (uint64_t)P->ns * sizeof(S), (uint32_t)Wb, 1);
        const bool ok2 = encode_tensor_map_2d(&tm_phi, dtp, P->d_PhiP, (uint64_t)P->MP, (uint64_t)P->K,
                                              (uint64_t)P->MP * sizeof(T), (uint32_t)P->MP, (uint32_t)kAdjP);
        use_tma = (ok1 && ok2) ? 1 : 0;
    }
    auto kern = adj_kernel<S, T, M>;
    {
        dr_status s = allow_dynamic_smem((const void *)kern, smem);
        if (s != DR_OK) return s;
    }
    const int ntx = (P->nx + TX - 1) / TX, nty = (P->ny + kAdjTY - 1) / kAdjTY;
    dim3 grid(ntx * nty, P->nz);
    kern<<<grid, kAdjThreads, smem, st>>>(tm_g, tm_phi, (const S *)g, (const T *)P->d_PhiP, P->d_adj,
                                          u_calc ? nullptr : (S *)u, u_calc ? (T *)u : nullptr, P->nx, P->ny,
                                          P->ns, P->K, P->m, P->MP, Wb, wbs, use_tma, (T)alpha, (T)beta,
                                          P->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adj_kernel launch");
    return DR_OK;
}


// Per-precision entry points (instantiated in projector_<prec>.cu).
template <typename S, typename T>
struct ProjOps {
    static dr_status fwd(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                         cudaStream_t st);
    static dr_status adj(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                         cudaStream_t st);
};

#define DR_DISPATCH_M(FN, S, T, ...)                      \
    switch (P->M) {                                       \
        case 1: return FN<S, T, 1>(__VA_ARGS__);          \
        case 2: return FN<S, T, 2>(__VA_ARGS__);          \
        case 4: return FN<S, T, 4>(__VA_ARGS__);          \
        case 8: return FN<S, T, 8>(__VA_ARGS__);          \
        case 12: return FN<S, T, 12>(__VA_ARGS__);        \
        case 16: return FN<S, T, 16>(__VA_ARGS__);        \
        case 24: return FN<S, T, 24>(__VA_ARGS__);        \
        case 32: return FN<S, T, 32>(__VA_ARGS__);        \
        default: return fail(DR_EINVAL, "unsupported m"); \
    }

template <typename S, typename T>
dr_status ProjOps<S, T>::fwd(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                             cudaStream_t st) {
    DR_DISPATCH_M(fwd_launch_t, S, T, P, u, out, gm, mode, sigma, st)
}

template <typename S, typename T>
dr_status ProjOps<S, T>::adj(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                             cudaStream_t st) {
    DR_DISPATCH_M(adj_launch_t, S, T, P, g, u, alpha, beta, u_calc, st)
}

extern template struct ProjOps<float, float>;
extern template struct ProjOps<bf16, float>;
extern template struct ProjOps<double, double>;

}  // namespace dr
