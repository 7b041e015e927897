// fold_impl.cuh -- half-turn folded projector pair (Sec. 4).
//
// With theta = n pi + theta0, theta0 in [0, pi), the static transform obeys
// R f(n pi + theta0, s) = R f(theta0, (-1)^n s) (exact for the Joseph
// discretisation on the symmetric bin grid).  Projections that share theta0
// (one per half-turn in a continuous scan) therefore need the static
// transform of each coefficient volume only once:
//
//   forward  g[k](s) = sum_j phi_j(t_k) (R u_j)(theta0_k, (-1)^{n_k} s)
//   adjoint  u_j = sum_{theta0} R*( gt_j(theta0) ),
//            gt_j(theta0, s) = sum_{k: theta0_k = theta0} phi_j(t_k) g[k]((-1)^{n_k} s)
//
// The forward marches the Joseph rays of each unique angle through a strip
// of the m-vector image staged in shared memory (all m coefficient sums per
// ray in registers) and distributes every ray to all projections of its
// angle in the epilogue.  The adjoint first folds the data per unique angle
// (fold_data_kernel, HBM bound), then back-projects the m folded sinograms
// with the voxel-driven exact transpose: per unique angle a TMA tile load of
// the footprint window (Wb bins x MS coefficients), mbarrier pipeline.
// Work per application drops from K (m + c) to U (2m + c') per voxel, U the
// number of unique angles.
#pragma once
#include <type_traits>

#include "dr_device.cuh"

namespace dr {

constexpr int kFoldThreads = 256;
constexpr int kFoldAdjP = 8;       // unique angles per adjoint pipeline stage (default; at most 32)
constexpr int kFoldAdjStages = 2;

// Padded coefficient stride in shared memory and in the folded data:
// multiples of 4 floats (16-byte vectors, TMA rows) whose pattern of
// 16-byte slots repeats only every 8 pixels (no bank conflicts between
// neighbouring pixels).
__host__ __device__ constexpr int fold_ms(int M) { return M <= 4 ? 4 : ((M % 8 == 0) ? M + 4 : M); }
__host__ __device__ constexpr int fold_rpt(int M) { return M <= 4 ? 8 : 32 / M; }

// Static-transform CTAs of the two-kernel forward (configurations in
// dr_internal.cuh): 1024 to 4096 rays per CTA.  The more rays a CTA carries,
// the more samples share each staged line.
// Strip element stride of a static group: 4 or 12 floats (bf16: 4 or 8).
__host__ __device__ constexpr int fold_static_ps(int MC, bool bf16) {
    return bf16 ? (MC == 4 ? 4 : 8) : (MC == 4 ? 4 : 12);
}

// Element stride of one pixel's coefficient vector in the forward strip.
// Float strips use fold_ms.  BF16 plans stage the stored bf16 values as they
// are (exact; the march widens them to float in registers), which halves the
// shared-memory bytes per ray step: 8-byte vectors for M <= 4, otherwise an
// odd number of 16-byte slots per pixel (no bank conflicts between
// neighbouring pixels).
__host__ __device__ constexpr int fold_bf16_ps(int M) {
    return M <= 4 ? 4 : 8 * (((M + 7) / 8) % 2 == 1 ? (M + 7) / 8 : (M + 7) / 8 + 1);
}
template <typename S, typename T, int M>
__host__ __device__ constexpr int fold_strip_ps() {
    return sizeof(S) == 2 ? fold_bf16_ps(M) : fold_ms(M);
}

// M bf16 coefficients of one strip pixel (PS-element slots), widened to float.
template <int M, int PS>
__device__ __forceinline__ void load_vec_bf16(const bf16 *p, float (&v)[M]) {
    if constexpr (PS == 4) {
        const uint2 a = *reinterpret_cast<const uint2 *>(p);
        const unsigned w[2] = {a.x, a.y};
#pragma unroll
        for (int j = 0; j < M; ++j) v[j] = __uint_as_float((j & 1) ? (w[j >> 1] & 0xffff0000u) : (w[j >> 1] << 16));
    } else {
#pragma unroll
        for (int c = 0; c < (M + 7) / 8; ++c) {
            const uint4 a = reinterpret_cast<const uint4 *>(p)[c];
            const unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int j = 8 * c + h;
                if (j < M) v[j] = __uint_as_float((h & 1) ? (w[h >> 1] & 0xffff0000u) : (w[h >> 1] << 16));
            }
        }
    }
}

template <typename T, int M>
__device__ __forceinline__ void load_vec(const T *p, T (&v)[M]) {
    if constexpr (sizeof(T) == 4 && (M % 4) == 0) {
#pragma unroll
        for (int j = 0; j < M / 4; ++j) {
            const float4 a = reinterpret_cast<const float4 *>(p)[j];
            v[4 * j] = a.x;
            v[4 * j + 1] = a.y;
            v[4 * j + 2] = a.z;
            v[4 * j + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < M; ++j) v[j] = p[j];
    }
}

// Copy the coefficients j0 .. j0+count-1 of one pixel (src points at j0) into
// the forward strip: bf16 strips keep the stored values, float strips hold
// the compute type; slots >= count are zero.  vec: src is 16-byte aligned
// and count == M, so whole 16-byte vectors may be moved (async_stage: with
// cp.async).
template <typename S, typename T, int M, typename ST>
__device__ __forceinline__ void stage_pixel(ST *dst, const S *__restrict__ src, int count, bool vec,
                                            int async_stage) {
    if constexpr (sizeof(S) == 2 && sizeof(ST) == 2) {
        if constexpr ((M % 8) == 0) {
            if (vec) {
                if (async_stage) {
#pragma unroll
                    for (int j = 0; j < M / 8; ++j) cp_async_16(dst + 8 * j, src + 8 * j);
                } else {
#pragma unroll
                    for (int j = 0; j < M / 8; ++j)
                        reinterpret_cast<uint4 *>(dst)[j] = __ldg(reinterpret_cast<const uint4 *>(src) + j);
                }
                return;
            }
        }
#pragma unroll
        for (int j = 0; j < M; ++j) dst[j] = j < count ? src[j] : S(0.0f);
    } else {
        T v[M];
        if constexpr (sizeof(S) == 4 && (M % 4) == 0) {
            if (vec) {
                if (async_stage) {
#pragma unroll
                    for (int j = 0; j < M / 4; ++j) cp_async_16(dst + 4 * j, src + 4 * j);
                    return;
                }
#pragma unroll
                for (int j = 0; j < M / 4; ++j) {
                    const float4 a = __ldg(reinterpret_cast<const float4 *>(src) + j);
                    v[4 * j] = a.x;
                    v[4 * j + 1] = a.y;
                    v[4 * j + 2] = a.z;
                    v[4 * j + 3] = a.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j) v[j] = j < count ? ldc<T>(src + j) : T(0);
            }
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) v[j] = j < count ? ldc<T>(src + j) : T(0);
        }
        if constexpr (sizeof(T) == 4 && (M % 4) == 0) {
#pragma unroll
            for (int j = 0; j < M / 4; ++j)
                reinterpret_cast<float4 *>(dst)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) dst[j] = v[j];
        }
    }
}

// ===========================================================================
// Forward
// ===========================================================================
// Resident CTAs per SM the folded forward asks the compiler for: the march is
// latency bound, and at M = 8 three CTAs (<= 85 registers) beat two.
__host__ __device__ constexpr int fold_fwd_min_blocks(int M) { return M == 8 ? 3 : 1; }

// STATIC = false: M covers all coefficients and the epilogue distributes each
// ray to the projections of its angle.  STATIC = true: the CTA handles the
// coefficient group j0 = (blockIdx.y % ngroups) * M .. j0 + M - 1 and writes
// the scaled static transforms (R u_j)(theta0_a, s_b) to
// ru[((z U + a) ns + b) ms_ru + j]; fold_dist_kernel distributes them.  With
// nsplit > 1 the march is split into nsplit chunks of image lines
// (blockIdx.z); chunk c writes its partial sums at ru + c * split_stride.
template <typename S, typename T, int M, bool STATIC, int THREADS = kFoldThreads, int RPTS = 0, int MINB = 1,
          bool TMA = false>
__global__ void __launch_bounds__(THREADS, THREADS == kFoldThreads ? fold_fwd_min_blocks(M) : MINB)
    fold_fwd_kernel(const S *__restrict__ u, S *__restrict__ out, const S *__restrict__ gm,
                    const FwdProj *__restrict__ uproj, const int *__restrict__ start, const int *__restrict__ member,
                    const T *__restrict__ phip, const int *__restrict__ blocks, int nx, int ny, int ns, int K,
                    int m, int MP, int P, int R, int nchunk, int mode, T sigma, int async_stage, int ngroups,
                    T *__restrict__ ru, int U, int ms_ru, int nsplit, size_t split_stride,
                    const __grid_constant__ CUtensorMap tm_rows, const __grid_constant__ CUtensorMap tm_cols,
                    int *status) {
    // strip element: stored bf16 for bf16 storage, else the compute type
    constexpr bool BF16_STRIP = sizeof(S) == 2;
    using ST = std::conditional_t<BF16_STRIP, S, T>;
    // TMA (static transforms of float coefficient groups of 4 or 8, staging
    // mode 3): strips staged by TMA into two buffers on mbarriers, in the TMA
    // line layout, each 4-coefficient plane of a group a line layout of its
    // own (16-byte entries: the even/odd halves stay conflict free); a
    // separate instantiation, so the other kernels carry none of its code
    constexpr bool TMA_CAP = TMA && STATIC && !BF16_STRIP && (M == 4 || M == 8);
    constexpr int NP = TMA_CAP ? M / 4 : 1;  // 16-byte planes per pixel (TMA strips)
    constexpr int MS = TMA_CAP ? 4 : (STATIC ? fold_static_ps(M, BF16_STRIP) : fold_strip_ps<S, T, M>());
    constexpr int RPT = STATIC ? RPTS : fold_rpt(M);
    constexpr int VW = 16 / (int)sizeof(S);  // elements per 16-byte vector
    extern __shared__ __align__(16) unsigned char fold_smem[];
    T *scale_s = reinterpret_cast<T *>(fold_smem);                       // [64]

    const int tid = threadIdx.x;
    const int z = blockIdx.y / ngroups;
    const int j0 = (blockIdx.y - z * ngroups) * M;
    const int count = min(M, m - j0);
    const bool vec = count == M && (m % VW) == 0 && (j0 % VW) == 0;
    const int blk_id = blockIdx.x / nchunk, chunk = blockIdx.x - blk_id * nchunk;
    const int *blk = blocks + (size_t)blk_id * P;
    const int branch = uproj[blk[0]].branch;
    const int W = branch ? ny : nx;
    const int H = branch ? nx : ny;
    constexpr bool tma = TMA_CAP;
    // line stride, zero entries before the even half, offset of the odd half
    // (TMA strips: a line is NP planes of fold_tma_line(W) entries each)
    const int ls = tma ? NP * fold_tma_line(W) : fold_line_elems(W);
    const int kg = tma ? 8 : kFoldGuardE;
    const int ooff = tma ? fold_tma_half(W) + 8 : fold_odd_off(W);
    ST *strip = reinterpret_cast<ST *>(
        tma ? fold_smem + 768 + ((128u - ((smem_u32(fold_smem) + 768u) & 127u)) & 127u) : fold_smem + 768);
    // image lines of this CTA's march: all, or chunk blockIdx.z of nsplit
    const int L0 = STATIC ? (int)(((long long)blockIdx.z * H) / nsplit) : 0;
    const int L1 = STATIC ? (int)(((long long)(blockIdx.z + 1) * H) / nsplit) : H;

    for (int p = tid; p < P; p += THREADS) {
        const int a = blk[p];
        const FwdProj f = uproj[a >= 0 ? a : blk[0]];
        scale_s[p] = (T)f.scale;
    }
    // strip buffers: 1 (synchronous staging), 2 (async_stage 1) or 3 (async_stage 2, 3)
    const int nbuf = tma ? kFoldTmaStages : async_stage + 1;
    if (tma) {
        // zero the guard entries only: TMA writes every data entry of a strip
        // (zero beyond the image), so no entry is written by both proxies
        const int wh = fold_tma_half(W), lp = fold_tma_line(W);  // plane line: 24 guard entries
        for (int i = tid; i < nbuf * R * NP * 24; i += THREADS) {
            const int pl = i / 24, g = i - pl * 24;  // pl: (buffer, line, plane)
            const int e = g < 8 ? g : (g < 16 ? kg + wh + (g - 8) : kg + ooff + wh + (g - 16));
            reinterpret_cast<float4 *>(strip)[(size_t)pl * lp + e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        for (int i = tid; i < nbuf * R * ls * MS; i += THREADS) strip[i] = ST(0.0f);
    }

    // Ray slots: thread t marches RPT rays of one distinct angle p_t of the
    // block, the bins l_t + tpa q (q = 0 .. RPT-1), so the rays of a thread
    // share their per-line step and consecutive threads take consecutive
    // bins; a single angle whose bins exceed one CTA (nchunk > 1) is cut into
    // chunks of THREADS * RPT bins, bins chunk * THREADS * RPT + t + THREADS q.
    const int tpa = nchunk > 1 ? THREADS : (ns + RPT - 1) / RPT;
    const int pt = nchunk > 1 ? 0 : tid / tpa;
    const int bt0 = nchunk > 1 ? chunk * THREADS * RPT + tid : tid - pt * tpa;
    const int at = pt < P ? blk[pt] : -1;
    long long xq[RPT];  // 32.32 position of each ray on its next line
    long long bfx = 0;  // per-line step of this thread's angle
    int lo[RPT], hi[RPT];
    unsigned rng[RPT];
    T acc[RPT][M];
    FwdProj f{};
    if (at >= 0) {
        f = uproj[at];
        bfx = f.B_fx;
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        lo[q] = 1;
        hi[q] = 0;
        xq[q] = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) acc[q][j] = T(0);
        const int b = bt0 + tpa * q;
        if (at >= 0 && b < ns) {
            xq[q] = f.C_fx + (long long)b * f.A_fx + (long long)L0 * bfx;
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
            lo[q] = max(lo[q], L0);
            hi[q] = min(hi[q], L1 - 1);
        }
        // the TMA kernel keeps each ray's line range in one register (lines < 2^16)
        rng[q] = (unsigned)lo[q] | ((unsigned)hi[q] << 16);
    }
    __syncthreads();

    const size_t zoff = (size_t)z * ny * nx;
    // Stage lines [r0, r0+nl) of the m-vector image into buffer `buf`:
    // asynchronously (cp.async, 16-byte chunks) when the coefficients are
    // 16-byte float vectors, else through registers.
    auto stage = [&](ST *buf, int r0, int nl) {
        const int npx = nl * W;
        for (int qq = tid; qq < npx; qq += THREADS) {
            int rl, i;
            size_t pix;
            if (branch == 0) {
                rl = qq / W;
                i = qq - rl * W;
                pix = zoff + (size_t)(r0 + rl) * nx + i;
            } else {
                i = qq / nl;
                rl = qq - i * nl;
                pix = zoff + (size_t)i * nx + (r0 + rl);
            }
            stage_pixel<S, T, M>(buf + ((size_t)rl * ls + (i & 1) * ooff + kg + (i >> 1)) * MS,
                                 u + pix * m + j0, count, vec, async_stage);
        }
    };
    const size_t buf_elems = (size_t)R * ls * MS;  // buffer b starts at strip + b * buf_elems
    if (!TMA_CAP && async_stage == 1 && L0 < L1) {
        stage(strip, L0, min(R, L1 - L0));
        cp_async_commit();
    }
    if (!TMA_CAP && async_stage == 2) {
        // three buffers: strips s+1 and s+2 are copied while strip s is marched,
        // and one barrier per strip suffices (the buffer refilled after the
        // barrier of strip s held strip s-1, which every thread has finished);
        // one commit group per strip, empty ones included, so that waiting for
        // all but the newest group always means strip s has landed
        if (L0 < L1) stage(strip, L0, min(R, L1 - L0));
        cp_async_commit();
        if (L0 + R < L1) stage(strip + buf_elems, L0 + R, min(R, L1 - L0 - R));
        cp_async_commit();
    }
    // ---- march the rays of lines [r0, r0 + nl) staged at cur: all m coefficient
    // sums per ray, line by line, the thread's RPT rays side by side
    // (independent chains); each ray still adds its lines in increasing order
    const int pstride = tma ? fold_tma_line(W) : 0;  // entries between the planes of a TMA line
    auto march = [&](const ST *cur, int r0, int nl) {
#pragma unroll 1
        for (int rl = 0; rl < nl; ++rl) {
            const int r = r0 + rl;
            const ST *row = cur + ((size_t)rl * ls + kg) * MS;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const int lq = TMA_CAP ? (int)(rng[q] & 0xffffu) : lo[q], hq = TMA_CAP ? (int)(rng[q] >> 16) : hi[q];
                if (r >= lq && r <= hq) {
                    const long long x = xq[q];
                    int i0 = (int)(x >> 32);
                    i0 = min(max(i0, -2), W);
                    const float w = __uint_as_float(0x3F800000u | ((unsigned)x >> 9)) - 1.0f;
                    const float w1m = 1.0f - w;
                    // pixels i0 and i0 + 1: the even one from the even half, the
                    // odd one from the odd half, each with its interpolation weight
                    const bool odd = i0 & 1;
                    const float we = odd ? w : w1m, wo = odd ? w1m : w;
                    const ST *pe = row + ((i0 + 1) >> 1) * MS, *po = row + (ooff + (i0 >> 1)) * MS;
                    T t0[M], t1[M];
                    if constexpr (BF16_STRIP) {
                        load_vec_bf16<M, MS>(pe, t0);
                        load_vec_bf16<M, MS>(po, t1);
                    } else if constexpr (NP > 1) {
                        // 4 coefficients per plane; plane p of the line pstride entries on
#pragma unroll
                        for (int pl = 0; pl < NP; ++pl) {
                            const float4 a = *reinterpret_cast<const float4 *>(pe + (size_t)pl * pstride * MS);
                            const float4 c = *reinterpret_cast<const float4 *>(po + (size_t)pl * pstride * MS);
                            t0[4 * pl] = a.x; t0[4 * pl + 1] = a.y; t0[4 * pl + 2] = a.z; t0[4 * pl + 3] = a.w;
                            t1[4 * pl] = c.x; t1[4 * pl + 1] = c.y; t1[4 * pl + 2] = c.z; t1[4 * pl + 3] = c.w;
                        }
                    } else {
                        load_vec<T, M>(pe, t0);
                        load_vec<T, M>(po, t1);
                    }
#pragma unroll
                    for (int j = 0; j < M; ++j) acc[q][j] = fmaf(wo, t1[j], fmaf(we, t0[j], acc[q][j]));
                }
                xq[q] += bfx;
            }
        }
    };
    if constexpr (TMA_CAP) {
        // Two strip buffers; full[b] completes when a strip's TMA copies have
        // landed (expect_tx).  One CTA barrier per strip: thread 0 waits for
        // strip s, the barrier then also says every thread has finished strip
        // s - 1, whose buffer the copies of strip s + 1 refill while strip s is
        // marched.  The copies of a strip are spread over the CTA's threads.
        // Waits are bounded: on a give-up the status word
        // is set and the CTA leaves in order.
        __shared__ __align__(8) uint64_t full[kFoldTmaStages];
        const int nstrips = L1 > L0 ? (L1 - L0 + R - 1) / R : 0;
        const size_t buf_elems = (size_t)R * ls * MS;
        if (tid == 0) {
            for (int b = 0; b < kFoldTmaStages; ++b) mbar_init(&full[b], 1);
            fence_mbar_init();
        }
        __syncthreads();
        // strip sidx into buffer sidx % 2: copy c of its 2 * nbox * nl by thread c (mod THREADS)
        auto issue = [&](int sidx) {
            const int b = sidx % kFoldTmaStages, r0s = L0 + sidx * R, nls = min(R, L1 - r0s);
            const int bw = fold_tma_bw(W), nbox = fold_tma_nbox(W), per_line = NP * 2 * nbox;
            if (tid == 0) mbar_arrive_expect_tx(&full[b], (unsigned)(nls * per_line * (bw / 2) * 16));
            for (int c = tid; c < nls * per_line; c += THREADS) {
                // copy c: line rl, plane pl (coefficients j0 + 4 pl ..), half, box bx
                const int rl = c / per_line, rem = c - rl * per_line, pl = rem / (2 * nbox),
                          rem2 = rem - pl * 2 * nbox, half = rem2 / nbox, bx = rem2 - half * nbox;
                const uint32_t dst = smem_u32(strip + b * buf_elems) +
                                     (uint32_t)(rl * ls + pl * pstride + kg + half * ooff + bx * (bw / 2)) * 16u;
                const int line = r0s + rl, p0 = bx * bw + half;
                if (branch == 0) tma_load_4d(dst, &tm_rows, j0 + 4 * pl, p0, line, z, &full[b]);
                else tma_load_4d(dst, &tm_cols, j0 + 4 * pl, line, p0, z, &full[b]);
            }
        };
        if (nstrips > 0) issue(0);
        for (int sidx = 0; sidx < nstrips; ++sidx) {
            const int b = sidx % kFoldTmaStages;
            int ok = 1;
            if (tid == 0) ok = mbar_wait_bounded_any(&full[b], (unsigned)((sidx / kFoldTmaStages) & 1), status,
                                                     2000000000ull);
            if (__syncthreads_or(!ok)) {
                // strip sidx did not land in time; let no copy of it outlive the CTA
                if (tid == 0)
                    mbar_wait_bounded(&full[b], (unsigned)((sidx / kFoldTmaStages) & 1), status, 100000000ull);
                return;
            }
            if (sidx + 1 < nstrips) issue(sidx + 1);
            const int r0 = L0 + sidx * R;
            march(strip + b * buf_elems, r0, min(R, L1 - r0));
        }
    }
    if constexpr (!TMA_CAP) {
        int s_idx = 0;
        for (int r0 = L0; r0 < L1; r0 += R, ++s_idx) {
            const int nl = min(R, L1 - r0);
            ST *cur;
            if (async_stage == 2) {
                cp_async_wait<1>();
                __syncthreads();
                if (r0 + 2 * R < L1) stage(strip + ((s_idx + 2) % 3) * buf_elems, r0 + 2 * R, min(R, L1 - r0 - 2 * R));
                cp_async_commit();
                cur = strip + (s_idx % 3) * buf_elems;
            } else if (async_stage) {
                // prefetch the next strip into the other buffer, then wait for this one
                if (r0 + R < L1) {
                    stage(strip + ((s_idx + 1) & 1) * buf_elems, r0 + R, min(R, L1 - r0 - R));
                    cp_async_commit();
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
                cur = strip + (s_idx & 1) * buf_elems;
            } else {
                stage(strip, r0, nl);
                __syncthreads();
                cur = strip;
            }
            march(cur, r0, nl);
            if (async_stage != 2) __syncthreads();
        }
        if (async_stage == 2) cp_async_wait<0>();  // no copy outlives the CTA
    }

    if constexpr (STATIC) {
        // ---- epilogue: the scaled static transforms of this coefficient group ----
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
            const int b = bt0 + tpa * q;
            const int a = at;
            if (a < 0 || b >= ns) continue;
            const T sc = scale_s[pt];
            T *dst = ru + blockIdx.z * split_stride + (((size_t)z * U + a) * ns + b) * ms_ru + j0;
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (j < count) dst[j] = sc * acc[q][j];
        }
        return;
    }
    // ---- epilogue: distribute each ray to every projection of its angle ----
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int b = bt0 + tpa * q;
        const int a = at;
        if (a < 0 || b >= ns) continue;
        const T sc = scale_s[pt];
        const int e = start[a + 1];
        for (int idx = start[a]; idx < e; ++idx) {
            const int mem = member[idx];
            const int k = mem >> 1;
            const int bb = (mem & 1) ? (ns - 1 - b) : b;
            const T *ph = phip + (size_t)k * MP;
            T val = T(0);
#pragma unroll
            for (int j = 0; j < M; ++j) val = fmaf(__ldg(ph + j), acc[q][j], val);
            val *= sc;
            const size_t o = ((size_t)z * K + k) * ns + bb;
            if (mode == 0) {
                stc<T>(out + o, val);
            } else if (mode == 1) {
                stc<T>(out + o, val - ldc<T>(gm + o));
            } else {
                const T h = ldc<T>(out + o);
                stc<T>(out + o, (h + sigma * val - sigma * ldc<T>(gm + o)) / (T(1) + sigma));
            }
        }
    }
}

// ===========================================================================
// Forward, two-kernel form, step 2: distribute the static transforms
//   g[z][k][b] = sum_j phi_j(t_k) ru[z][a(k)][flip_k(b)][j]
// with the forward epilogue modes (store, minus gm, CP dual update).  Line
// chunks of a split march are added first, in chunk order.  A thread takes
// one row (z, a, b) of the static transforms, reads it once, and writes the
// bins of every projection k of angle a (at b, or ns-1-b for odd half-turns):
// consecutive threads write consecutive bins of the same projection.
// ===========================================================================
template <typename S, typename T, int M>
__global__ void __launch_bounds__(kRedThreads)
    fold_dist_kernel(const T *__restrict__ ru, S *__restrict__ out, const S *__restrict__ gm,
                     const int *__restrict__ start, const int *__restrict__ member, const T *__restrict__ phip,
                     int nz, int K, int ns, int U, int ms_ru, int m, int MP, int mode, T sigma, int nsplit,
                     size_t split_stride) {
    // rows and table rows are multiples of 4 floats from 16-byte aligned bases
    constexpr bool V4 = sizeof(T) == 4;
    const size_t n = (size_t)nz * U * ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i % ns);
        const size_t za = i / ns;
        const int a = (int)(za % U), z = (int)(za / U);
        const T *r = ru + i * ms_ru;
        T rv[M];
        if constexpr (V4 && M % 4 == 0) {
#pragma unroll
            for (int q = 0; q < M / 4; ++q) {
                if (4 * q < m) {
                    float4 v = *reinterpret_cast<const float4 *>(r + 4 * q);
                    for (int c = 1; c < nsplit; ++c) {
                        const float4 w = *reinterpret_cast<const float4 *>(r + c * split_stride + 4 * q);
                        v.x += w.x;
                        v.y += w.y;
                        v.z += w.z;
                        v.w += w.w;
                    }
                    rv[4 * q] = v.x;
                    rv[4 * q + 1] = v.y;
                    rv[4 * q + 2] = v.z;
                    rv[4 * q + 3] = v.w;
                } else {
                    rv[4 * q] = rv[4 * q + 1] = rv[4 * q + 2] = rv[4 * q + 3] = T(0);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                T rj = T(0);
                if (j < m) {
                    rj = r[j];
                    for (int c = 1; c < nsplit; ++c) rj += r[c * split_stride + j];
                }
                rv[j] = rj;
            }
        }
        const int e = __ldg(start + a + 1);
        for (int idx = __ldg(start + a); idx < e; ++idx) {
            const int mem = __ldg(member + idx);
            const int k = mem >> 1;
            const int bb = (mem & 1) ? ns - 1 - b : b;
            const T *ph = phip + (size_t)k * MP;
            T val = T(0);
            if constexpr (V4 && M % 4 == 0) {
#pragma unroll
                for (int q = 0; q < M / 4; ++q) {
                    if (4 * q >= m) break;
                    const float4 f = __ldg(reinterpret_cast<const float4 *>(ph) + q);
                    const float fv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (4 * q + t < m) val = fma(fv[t], rv[4 * q + t], val);
                }
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j)
                    if (j < m) val = fma(__ldg(ph + j), rv[j], val);
            }
            const size_t o = ((size_t)z * K + k) * ns + bb;
            if (mode == 0) {
                stc<T>(out + o, val);
            } else if (mode == 1) {
                stc<T>(out + o, val - ldc<T>(gm + o));
            } else {
                const T h = ldc<T>(out + o);
                stc<T>(out + o, (h + sigma * val - sigma * ldc<T>(gm + o)) / (T(1) + sigma));
            }
        }
    }
}

// ===========================================================================
// Adjoint, step 1: fold the data per unique angle
//   gt[z][a][b][j] = sum_{k in group(a)} phi_j(t_k) g[z][k][flip_k(b)]
// ===========================================================================
template <typename S, typename T, int M>
__global__ void __launch_bounds__(kRedThreads)
    fold_data_kernel(const S *__restrict__ g, T *__restrict__ gt, const int *__restrict__ start,
                     const int *__restrict__ member, const T *__restrict__ phip, int nz, int U, int ns, int K, int MP) {
    constexpr int MS = fold_ms(M);
    const size_t n = (size_t)nz * U * ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(i % ns);
        const size_t r = i / ns;
        const int a = (int)(r % U);
        const int z = (int)(r / U);
        T acc[M];
#pragma unroll
        for (int j = 0; j < M; ++j) acc[j] = T(0);
        const int e = __ldg(start + a + 1);
        // members in groups of 4: their data loads are issued together (the
        // accumulation keeps the member order)
        constexpr int G = 4;
        for (int idx0 = __ldg(start + a); idx0 < e; idx0 += G) {
            int kq[G];
            T gv[G];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const int idx = idx0 + q;
                const int mem = idx < e ? __ldg(member + idx) : 0;
                kq[q] = mem >> 1;
                const int bb = (mem & 1) ? (ns - 1 - b) : b;
                gv[q] = idx < e ? ldc<T>(g + ((size_t)z * K + kq[q]) * ns + bb) : T(0);
            }
#pragma unroll
            for (int q = 0; q < G; ++q) {
                if (idx0 + q >= e) break;
                const T *ph = phip + (size_t)kq[q] * MP;
                if constexpr (sizeof(T) == 4 && M % 4 == 0) {
#pragma unroll
                    for (int c = 0; c < M / 4; ++c) {
                        const float4 f = __ldg(reinterpret_cast<const float4 *>(ph) + c);
                        acc[4 * c] = fmaf(f.x, gv[q], acc[4 * c]);
                        acc[4 * c + 1] = fmaf(f.y, gv[q], acc[4 * c + 1]);
                        acc[4 * c + 2] = fmaf(f.z, gv[q], acc[4 * c + 2]);
                        acc[4 * c + 3] = fmaf(f.w, gv[q], acc[4 * c + 3]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < M; ++j) acc[j] = fmaf(__ldg(ph + j), gv[q], acc[j]);
                }
            }
        }
        T *dst = gt + i * MS;
        if constexpr ((MS % 4) == 0 && sizeof(T) == 4) {
            float v[MS];
#pragma unroll
            for (int j = 0; j < MS; ++j) v[j] = j < M ? acc[j] : 0.0f;
#pragma unroll
            for (int j = 0; j < MS / 4; ++j)
                reinterpret_cast<float4 *>(dst)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < MS; ++j) dst[j] = j < M ? acc[j] : T(0);
        }
    }
}

// ===========================================================================
// Adjoint, step 2: voxel-driven exact transpose of the folded sinograms
// ===========================================================================
struct alignas(16) FoldPrm {
    float c, s, c8, qb;   // cos, sin, 8 cos, window-relative origin position - 1/2
    float e0, inv_c2;     // 1/c - 1/(2c^2), 1/c^2
    int idx_base;         // integer origin position minus the float magic
    float c16;            // 16 cos
};

// Tile of TX x kAdjTY voxels per CTA of 128 threads, VPT voxels per thread.
// PAIRED (VPT even): a thread holds voxel pairs (x, y), (x, y+1) in VPT/2
// columns x0 + tx + 16 v (threads 16 x 8, rows y0 + 2 ty + {0, 1}).  The two
// voxels of a pair project sin(theta) apart, so their taps lie in three
// consecutive bins: one read of three bins serves both (3 instead of 4 bin
// reads per voxel and angle).  Otherwise threads 8 x 16, columns x0 + tx + 8 v.
template <int M>
struct FoldAdjShape {
    static constexpr int VPT = (M <= 8) ? 4 : ((M <= 16) ? 2 : 1);
    static constexpr int TX = 8 * VPT;
    static constexpr bool PAIRED = (VPT % 2) == 0;
};

// Seven 128-thread CTAs per SM (<= 72 registers): with the default seven
// angles per pipeline stage, shared memory admits seven too (M <= 16).
__host__ __device__ constexpr int fold_adj_min_blocks(int M) { return M <= 16 ? 7 : 6; }

template <typename S, typename T, int M>
__global__ void __launch_bounds__(kAdjThreads, fold_adj_min_blocks(M))
    fold_adj_kernel(const __grid_constant__ CUtensorMap tm_gt, const AdjProj *__restrict__ uproj,
                    S *__restrict__ u_s, T *__restrict__ u_c, int nx, int ny, int U, int m, int Wb, T alpha, T beta,
                    int *status, int PP) {
    constexpr int VPT = FoldAdjShape<M>::VPT;
    constexpr int TX = FoldAdjShape<M>::TX;
    constexpr int TY = kAdjTY;
    constexpr int NST = kFoldAdjStages;
    constexpr int MS = fold_ms(M);
    constexpr float kMag = 12582912.0f;
    constexpr int kMagI = 0x4B400000;

    extern __shared__ __align__(128) unsigned char fadj_smem_raw[];
    // round up to 128 B by pointer arithmetic on the __shared__ array, so the
    // compiler keeps addressing it as shared memory (LDS, not generic loads)
    unsigned char *smem_raw = fadj_smem_raw + ((128u - (smem_u32(fadj_smem_raw) & 127u)) & 127u);
    const size_t row_bytes = ((size_t)Wb * MS * sizeof(T) + 127) & ~(size_t)127;
    const size_t win_bytes = PP * row_bytes;
    const size_t stage_bytes = win_bytes + 128 * ((PP * sizeof(FoldPrm) + 127) / 128);
    __shared__ __align__(8) uint64_t full[NST];
    auto win_s = [&](int st, int p) { return reinterpret_cast<T *>(smem_raw + st * stage_bytes + p * row_bytes); };
    auto prm_s = [&](int st) { return reinterpret_cast<FoldPrm *>(smem_raw + st * stage_bytes + win_bytes); };

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ntx = (nx + TX - 1) / TX;
    const int x0 = (blockIdx.x % ntx) * TX, y0 = (blockIdx.x / ntx) * TY;
    const int z = blockIdx.y;
    const int xo = x0 + TX / 2, yo = y0 + TY / 2;
    constexpr bool PAIRED = FoldAdjShape<M>::PAIRED;
    const int tx = PAIRED ? (tid & 15) : (tid & 7), ty = PAIRED ? (tid >> 4) : (tid >> 3);
    const int dx0 = x0 + tx - xo, dy = (PAIRED ? y0 + 2 * ty : y0 + ty) - yo;
    const int nkb = (U + PP - 1) / PP;

    auto issue = [&](int st, int kb) {
        int wb0 = 0, row = 0;
        if (lane < PP) {
            const int a = kb * PP + lane;
            const int aa = a < U ? a : U - 1;
            const AdjProj pj = uproj[aa];
            const double posO = xo * pj.c + yo * pj.s + pj.C0;
            const double emin = posO + fmin((-TX / 2) * pj.c, (TX / 2 - 1) * pj.c) +
                                fmin((-TY / 2) * pj.s, (TY / 2 - 1) * pj.s);
            wb0 = (int)floor(emin) - 1;
            const double rel = posO - wb0;
            const double ri = floor(rel);
            FoldPrm pr;
            pr.c = (float)pj.c;
            pr.s = (float)pj.s;
            pr.c8 = (float)(8.0 * pj.c);
            pr.qb = (float)(rel - ri) - 0.5f;
            pr.inv_c2 = (float)(pj.inv_c * pj.inv_c);
            pr.e0 = (float)(pj.inv_c - 0.5 * pj.inv_c * pj.inv_c);
            pr.idx_base = (int)ri - kMagI;
            pr.c16 = (float)(16.0 * pj.c);
            prm_s(st)[lane] = pr;
            row = z * U + aa;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_expect_tx(&full[st], (unsigned)(PP * Wb * MS * sizeof(T)));
        __syncwarp();
        if (lane < PP) tma_load_3d(win_s(st, lane), &tm_gt, 0, wb0, row, &full[st]);
        if (lane != 0) mbar_arrive(&full[st]);
    };

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&full[s], 32);
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == 0)
        for (int s = 0; s < NST && s < nkb; ++s) issue(s, s);

    T acc[VPT][M];
#pragma unroll
    for (int v = 0; v < VPT; ++v)
#pragma unroll
        for (int j = 0; j < M; ++j) acc[v][j] = T(0);

    const float dxf = (float)dx0, dyf = (float)dy;
    for (int kb = 0; kb < nkb; ++kb) {
        const int st = kb % NST;
        const bool bad = !mbar_wait_bounded(&full[st], (unsigned)((kb / NST) & 1), status, 2000000000ull);
        if (!bad) {
            const FoldPrm *prm = prm_s(st);
            const int np = min(PP, U - kb * PP);
            for (int p = 0; p < np; ++p) {
                const FoldPrm a = prm[p];
                const T *w = win_s(st, p);
                float q = fmaf(dyf, a.s, fmaf(dxf, a.c, a.qb));
                // Pairs need the two rows' taps within three bins: |qB - qA| < 1.
                // With |sin| <= 1 - 1e-5 and |q| < 64 (rounding of qA + sin below
                // 4e-6) the rounded bin indices differ by at most one; angles
                // closer to |sin| = 1 (a warp-uniform test) use the per-voxel path.
                if (PAIRED && fabsf(a.s) <= 0.99999f) {
#pragma unroll
                    for (int v = 0; v < VPT / 2; ++v) {
                        // rows y (A) and y + 1 (B) of column v
                        const float qA = q, qB = q + a.s;
                        const float tA = qA + kMag, tB = qB + kMag;
                        const float dA = qA - (tA - kMag), dB = qB - (tB - kMag);
                        const int iA = __float_as_int(tA) + a.idx_base, iB = __float_as_int(tB) + a.idx_base;
                        const float w0A = fmaxf(0.0f, fmaf(-dA, a.inv_c2, a.e0));
                        const float w1A = fmaxf(0.0f, fmaf(dA, a.inv_c2, a.e0));
                        const float w0B = fmaxf(0.0f, fmaf(-dB, a.inv_c2, a.e0));
                        const float w1B = fmaxf(0.0f, fmaf(dB, a.inv_c2, a.e0));
                        {
                            // taps iA, iA+1 and iB, iB+1 within bins b, b+1, b+2: each
                            // voxel's weights on the three bins (one of them an exact 0)
                            const int b = min(iA, iB);
                            const bool lA = iA == b, lB = iB == b;
                            const float oA0 = lA ? w0A : 0.0f, oA1 = lA ? w1A : w0A, oA2 = lA ? 0.0f : w1A;
                            const float oB0 = lB ? w0B : 0.0f, oB1 = lB ? w1B : w0B, oB2 = lB ? 0.0f : w1B;
                            const T *r0 = w + b * MS;
                            constexpr int CH = (M % 4) == 0 ? 4 : M;  // coefficients per chunk
#pragma unroll
                            for (int c0 = 0; c0 < M; c0 += CH) {
                                T b0[CH], b1[CH], b2[CH];
                                load_vec<T, CH>(r0 + c0, b0);
                                load_vec<T, CH>(r0 + MS + c0, b1);
                                load_vec<T, CH>(r0 + 2 * MS + c0, b2);
#pragma unroll
                                for (int j = 0; j < CH; ++j) {
                                    T &ra = acc[2 * v][c0 + j];
                                    ra = fmaf(oA2, b2[j], fmaf(oA1, b1[j], fmaf(oA0, b0[j], ra)));
                                    T &rb = acc[2 * v + 1][c0 + j];
                                    rb = fmaf(oB2, b2[j], fmaf(oB1, b1[j], fmaf(oB0, b0[j], rb)));
                                }
                            }
                        }
                        q += a.c16;
                    }
                    continue;
                }
                // one voxel at a time: voxel v at q (+ sin for the second row of a pair)
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const float qv = (PAIRED && (v & 1)) ? q + a.s : q;
                    const float t = qv + kMag;
                    const float fl = t - kMag;
                    const float d = qv - fl;
                    const int idx = __float_as_int(t) + a.idx_base;
                    const float w0 = fmaxf(0.0f, fmaf(-d, a.inv_c2, a.e0));
                    const float w1 = fmaxf(0.0f, fmaf(d, a.inv_c2, a.e0));
                    T t0[M], t1[M];
                    load_vec<T, M>(w + idx * MS, t0);
                    load_vec<T, M>(w + (idx + 1) * MS, t1);
#pragma unroll
                    for (int j = 0; j < M; ++j) acc[v][j] = fmaf(w1, t1[j], fmaf(w0, t0[j], acc[v][j]));
                    if (!PAIRED) q += a.c8;
                    else if (v & 1) q += a.c16;
                }
            }
        }
        if (__syncthreads_or(bad)) {
            if (tid == 0)
                for (int s = kb; s < nkb && s < kb + NST; ++s)
                    mbar_wait_bounded(&full[s % NST], (unsigned)((s / NST) & 1), status, 100000000ull);
            return;
        }
        if (warp == 0 && kb + NST < nkb) issue(st, kb + NST);
    }

#pragma unroll
    for (int v = 0; v < VPT; ++v) {
        const int x = PAIRED ? x0 + tx + 16 * (v >> 1) : x0 + tx + 8 * v;
        const int y = PAIRED ? y0 + 2 * ty + (v & 1) : y0 + ty;
        if (x >= nx || y >= ny) continue;
        const size_t base = (((size_t)z * ny + y) * nx + x) * m;
#pragma unroll
        for (int j = 0; j < M; ++j)
            if (j < m) {
                if (u_c) {
                    T r = alpha * acc[v][j];
                    if (beta != T(0)) r += beta * u_c[base + j];
                    u_c[base + j] = r;
                } else {
                    T r = alpha * acc[v][j];
                    if (beta != T(0)) r += beta * ldc<T>(u_s + base + j);
                    stc<T>(u_s + base + j, r);
                }
            }
    }
}

// ===========================================================================
// Host launchers
// ===========================================================================
inline int fold_adj_wb(int M) {
    const int VPT = (M <= 8) ? 4 : ((M <= 16) ? 2 : 1);
    const int TX = 8 * VPT;
    const double ext = std::sqrt((double)(TX - 1) * (TX - 1) + (double)(kAdjTY - 1) * (kAdjTY - 1));
    return (int)std::ceil(ext) + 6;
}

template <typename S, typename T, int M>
dr_status fold_fwd_launch_t(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                            cudaStream_t st) {
    using ST = std::conditional_t<sizeof(S) == 2, S, T>;
    constexpr int MS = fold_strip_ps<S, T, M>();
    const int ls = fold_line_elems_max(P->nx, P->ny);
    // strip height and staging mode: the autotuned choice (cp.async double
    // buffering needs whole 16-byte coefficient vectors)
    const int async_ok = (P->m == M && ((sizeof(S) == 4 && (M % 4) == 0) || (sizeof(S) == 2 && (M % 8) == 0))) ? 1 : 0;
    const bool bf16_strip = sizeof(S) == 2;
    const int async_stage = async_ok && (bf16_strip ? P->fold_async_st : P->fold_async);
    const int R = std::max(1, bf16_strip ? P->fold_lines_st : P->fold_lines);
    const size_t smem = 768 + sizeof(ST) * (size_t)(async_stage + 1) * R * ls * MS;
    auto kern = fold_fwd_kernel<S, T, M, false>;
    {
        dr_status s = allow_dynamic_smem((const void *)kern, smem);
        if (s != DR_OK) return s;
    }
    dim3 grid(P->n_fold_blocks * P->fold_nchunk, P->nz);
    kern<<<grid, kFoldThreads, smem, st>>>((const S *)u, (S *)out, (const S *)gm, P->d_fold_fwd, P->d_fold_start,
                                           P->d_fold_member, (const T *)P->d_PhiP, P->d_fold_blocks, P->nx, P->ny,
                                           P->ns, P->K, P->m, P->MP, P->fold_P, R, P->fold_nchunk, mode,
                                           (T)sigma, async_stage, 1, (T *)nullptr, 0, 0, 1, (size_t)0, CUtensorMap{},
                                           CUtensorMap{}, P->d_status);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DR_OK : cuda_fail(e, "fold_fwd_kernel launch");
}

// Two-kernel folded forward: static transforms of coefficient groups of MC
// (4 or 8) into the folded-data scratch, then the distribution.
// Static transforms of the two-kernel forward (step 1), into the folded-data
// scratch (one march) or the split scratch (line chunks); `rs` says where.
struct StaticOut {
    void *ru;
    int ms_ru, nsplit;
    size_t split_stride;
};

template <typename S, typename T, int M, int GI>
dr_status fold_static_launch(dr_plan *P, const void *u, cudaStream_t st, StaticOut &rs) {
    constexpr int MC = fold_static_mc(GI), THREADS = fold_static_threads(GI), RPT = fold_static_rpt_gi(GI),
                  MINB = fold_static_min_blocks(GI);
    constexpr bool BF16_STRIP = sizeof(S) == 2;
    using ST = std::conditional_t<BF16_STRIP, S, T>;
    constexpr int MS = fold_static_ps(MC, BF16_STRIP);
    constexpr int VW = 16 / (int)sizeof(S);
    const int gi = GI;
    const int ngroups = (P->m + MC - 1) / MC;
    const int ls = fold_line_elems_max(P->nx, P->ny);
    const bool bf16_kernel = sizeof(S) == 2;
    const int async_req = bf16_kernel ? P->fold2_async_st : P->fold2_async;
    const int R0 = std::max(1, std::min(bf16_kernel ? P->fold2_lines_st : P->fold2_lines,
                                        async_req == 3 && !bf16_kernel && P->fold2_Rt[gi] > 0 ? P->fold2_Rt[gi]
                                                                                              : P->fold2_R[gi]));
    if ((size_t)P->nz * ngroups > 65535) return fail(DR_EINVAL, "two-kernel folded forward: too many slice groups");
    // async 1: two strip buffers, the next strip copied with cp.async while the
    // current one is marched (groups of whole 16-byte vectors; other pixels
    // are staged through registers); async 2: three buffers, two strips ahead
    (void)VW;
    int async = bf16_kernel ? P->fold2_async_st : P->fold2_async;
    int R = R0;
    // async 3: TMA-staged strips (4-float groups of a float plan whose rows
    // of coefficients are whole 16-byte vectors); otherwise three cp.async buffers
    CUtensorMap tm_rows{}, tm_cols{};
    constexpr int NPT = MC / 4;  // 16-byte planes per pixel of a TMA strip
    if (async == 3) {
        bool ok = !BF16_STRIP && (P->m % 4) == 0 && ((uintptr_t)u % 16) == 0;
        if (ok) {
            const uint64_t dims[4] = {(uint64_t)P->m, (uint64_t)P->nx, (uint64_t)P->ny, (uint64_t)P->nz};
            const uint64_t strides[3] = {(uint64_t)P->m * 4, (uint64_t)P->nx * P->m * 4,
                                         (uint64_t)P->ny * P->nx * P->m * 4};
            const uint32_t box_r[4] = {4, (uint32_t)fold_tma_bw(P->nx), 1, 1}, es_r[4] = {1, 2, 1, 1};
            const uint32_t box_c[4] = {4, 1, (uint32_t)fold_tma_bw(P->ny), 1}, es_c[4] = {1, 1, 2, 1};
            ok = encode_tensor_map(&tm_rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(u), dims,
                                   strides, box_r, es_r) &&
                 encode_tensor_map(&tm_cols, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(u), dims,
                                   strides, box_c, es_c);
        }
        if (ok) {
            const long long line = 16LL * NPT * std::max(fold_tma_line(P->nx), fold_tma_line(P->ny));
            R = std::max(1, std::min(R, (int)((2LL * kFoldStripBudget) / (kFoldTmaStages * line))));
        } else {
            async = 2;
        }
    }
    if (async == 2) {
        // three buffers within twice the strip budget (below the 227 KB a CTA
        // may hold); where even one line does not fit, two buffers (same march)
        const long long line = (long long)sizeof(ST) * ls * MS;
        const int r3 = (int)((2LL * kFoldStripBudget) / (3 * line));
        if (r3 >= 1) R = std::min(R, r3);
        else async = 1;
    }
    const size_t smem = async == 3 ? 768 + 128 + 16 * (size_t)kFoldTmaStages * R * NPT *
                                               std::max(fold_tma_line(P->nx), fold_tma_line(P->ny))
                                   : 768 + sizeof(ST) * (size_t)(async + 1) * R * ls * MS;
    auto kern = fold_fwd_kernel<S, T, MC, true, THREADS, RPT, MINB>;
    if constexpr (!BF16_STRIP) {
        if (async == 3) kern = fold_fwd_kernel<S, T, MC, true, THREADS, RPT, MINB, true>;
    }
    {
        dr_status s = allow_dynamic_smem((const void *)kern, smem);
        if (s != DR_OK) return s;
    }
    // one march: static transforms into the folded-data scratch (row stride
    // fold_ms(M)); a march split into line chunks: partial sums into the
    // split scratch (row stride m rounded up to 4), one chunk after another
    const int nsplit = P->split_off ? 1 : std::max(1, P->fold2_split);
    T *ru;
    int ms_ru;
    size_t split_stride = 0;
    if (nsplit == 1) {
        dr_status s = ensure_fold_scratch(P);
        if (s != DR_OK) return s;
        ru = (T *)P->d_gt;
        ms_ru = fold_ms(M);
    } else {
        ms_ru = (P->m + 3) / 4 * 4;
        split_stride = (size_t)P->nz * P->fold_U * P->ns * ms_ru;
        dr_status s = ensure_split_scratch(P, sizeof(T) * split_stride * nsplit);
        if (s != DR_OK) return s;
        ru = (T *)P->d_ru_split;
    }
    const int bv = P->d_fold2_blocks[gi][P->fold2_bv] ? P->fold2_bv : 0;
    dim3 grid(P->fold2_nblocks[gi][bv] * P->fold2_nchunk[gi], P->nz * ngroups, nsplit);
    kern<<<grid, THREADS, smem, st>>>((const S *)u, (S *)nullptr, (const S *)nullptr, P->d_fold_fwd, P->d_fold_start,
                                           P->d_fold_member, (const T *)P->d_PhiP, P->d_fold2_blocks[gi][bv],
                                           P->nx, P->ny, P->ns, P->K, P->m, P->MP, P->fold2_P[gi][bv], R,
                                           P->fold2_nchunk[gi],
                                           0, (T)0, async, ngroups, ru, P->fold_U, ms_ru, nsplit,
                                           split_stride, tm_rows, tm_cols, P->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fold_fwd_kernel (static) launch");
    rs = StaticOut{ru, ms_ru, nsplit, split_stride};
    return DR_OK;
}

template <typename S, typename T, int M>
dr_status fold_static_dispatch(dr_plan *P, const void *u, cudaStream_t st, StaticOut &rs) {
    if (!P->fold2_ok) return fail(DR_EINVAL, "two-kernel folded forward unavailable for this plan");
    if constexpr (M >= 4) {
        switch (sizeof(S) == 2 ? P->fold2_gi_st : P->fold2_gi) {
            case 0: return fold_static_launch<S, T, M, 0>(P, u, st, rs);
            case 2: return fold_static_launch<S, T, M, 2>(P, u, st, rs);
            case 4: return fold_static_launch<S, T, M, 4>(P, u, st, rs);
            case 6: return fold_static_launch<S, T, M, 6>(P, u, st, rs);
            case 1:
                if constexpr (M >= 8) return fold_static_launch<S, T, M, 1>(P, u, st, rs);
                break;
            case 3:
                if constexpr (M >= 8) return fold_static_launch<S, T, M, 3>(P, u, st, rs);
                break;
            case 5:
                if constexpr (M >= 8) return fold_static_launch<S, T, M, 5>(P, u, st, rs);
                break;
            case 7:
                if constexpr (M >= 8) return fold_static_launch<S, T, M, 7>(P, u, st, rs);
                break;
        }
    }
    return fail(DR_EINVAL, "two-kernel folded forward: unsupported coefficient group");
}

template <typename S, typename T, int M>
dr_status fold_fwd2_launch_t(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                             cudaStream_t st) {
    StaticOut rs{};
    {
        dr_status s = fold_static_dispatch<S, T, M>(P, u, st, rs);
        if (s != DR_OK) return s;
    }
    fold_dist_kernel<S, T, M><<<red_grid((size_t)P->nz * P->fold_U * P->ns), kRedThreads, 0, st>>>(
        (const T *)rs.ru, (S *)out, (const S *)gm, P->d_fold_start, P->d_fold_member, (const T *)P->d_PhiP, P->nz,
        P->K, P->ns, P->fold_U, rs.ms_ru, P->m, P->MP, mode, (T)sigma, rs.nsplit, rs.split_stride);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DR_OK : cuda_fail(e, "fold_dist_kernel launch");
}

// gt: where the folded data live (nz U ns MS floats); nullptr: the plan's
// scratch buffer.
template <typename S, typename T, int M>
dr_status fold_backproject(dr_plan *P, void *u, double alpha, double beta, bool u_calc, cudaStream_t st,
                           void *gt = nullptr);

template <typename S, typename T, int M>
dr_status fold_adj_launch_t(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                            cudaStream_t st, void *gt = nullptr) {
    constexpr int MS = fold_ms(M);
    if (!gt) gt = P->d_gt;
    // step 1: fold the data into the scratch buffer
    fold_data_kernel<S, T, M><<<red_grid((size_t)P->nz * P->fold_U * P->ns), kRedThreads, 0, st>>>(
        (const S *)g, (T *)gt, P->d_fold_start, P->d_fold_member, (const T *)P->d_PhiP, P->nz, P->fold_U, P->ns,
        P->K, P->MP);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fold_data_kernel launch");
    return fold_backproject<S, T, M>(P, u, alpha, beta, u_calc, st, gt);
}

// Back-project the folded sinograms (step 2 of the folded adjoint):
// u = alpha R*(folded) + beta u.
template <typename S, typename T, int M>
dr_status fold_backproject(dr_plan *P, void *u, double alpha, double beta, bool u_calc, cudaStream_t st, void *gt) {
    constexpr int MS = fold_ms(M);
    if (!gt) gt = P->d_gt;
    const int Wb = fold_adj_wb(M);
    CUtensorMap tm{};
    const uint64_t dims[3] = {(uint64_t)MS, (uint64_t)P->ns, (uint64_t)P->nz * P->fold_U};
    const uint64_t strides[2] = {(uint64_t)MS * sizeof(T), (uint64_t)P->ns * MS * sizeof(T)};
    const uint32_t box[3] = {(uint32_t)MS, (uint32_t)Wb, 1};
    if (!encode_tensor_map(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, gt, dims, strides, box))
        return fail(DR_ECUDA, "fold adj: tensor map encode failed");
    // angles per pipeline stage: fewer shrink the windows' shared memory so that
    // more CTAs fit on an SM (the angles are summed in the same order)
    const int pp = std::max(1, std::min(32, P->fold_adj_pp));
    const size_t row_bytes = ((size_t)Wb * MS * sizeof(T) + 127) & ~(size_t)127;
    const size_t stage = pp * row_bytes + 128 * ((pp * sizeof(FoldPrm) + 127) / 128);
    const size_t smem = stage * kFoldAdjStages + 128;
    auto kern = fold_adj_kernel<S, T, M>;
    {
        dr_status s = allow_dynamic_smem((const void *)kern, smem);
        if (s != DR_OK) return s;
    }
    constexpr int TX = FoldAdjShape<M>::TX;
    const int ntx = (P->nx + TX - 1) / TX, nty = (P->ny + kAdjTY - 1) / kAdjTY;
    dim3 grid(ntx * nty, P->nz);
    kern<<<grid, kAdjThreads, smem, st>>>(tm, P->d_fold_adj, u_calc ? nullptr : (S *)u, u_calc ? (T *)u : nullptr,
                                          P->nx, P->ny, P->fold_U, P->m, Wb, (T)alpha, (T)beta, P->d_status, pp);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DR_OK : cuda_fail(e, "fold_adj_kernel launch");
}

// ===========================================================================
// Normal operator R*R of the folded pair, as the CG steps use it.  Per
// distinct angle a, forward then adjoint give
//   (R*R u)_i = sum_a R_a* [ sum_j G_a[i][j] (R_a u_j) ],
//   G_a = sum_{k in a} phi(t_k) phi(t_k)^T,
// because the bin reversal of an odd half-turn is undone by its adjoint.  So
// the static transforms are mixed by G_a per (slice, angle, bin) and
// back-projected, without the K projections in between.
// ===========================================================================
template <typename T, int M>
__global__ void __launch_bounds__(kRedThreads)
    fold_gram_kernel(const T *ru, T *gt, const T *__restrict__ gram, int nz, int U, int ns, int ms_ru, int m,
                     int nsplit, size_t split_stride) {
    // ru and gt may be the same buffer (one chunk): each thread reads its row
    // whole before writing it, so they are not declared __restrict__
    constexpr int MS = fold_ms(M);
    constexpr bool V4 = sizeof(T) == 4;
    const size_t n = (size_t)nz * U * ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)((i / ns) % U);
        const T *r = ru + i * ms_ru;
        T rv[M];
        if constexpr (V4 && M % 4 == 0) {
            // rows are multiples of 4 floats from 16-byte aligned bases
#pragma unroll
            for (int q = 0; q < M / 4; ++q) {
                if (4 * q < m) {
                    float4 v = *reinterpret_cast<const float4 *>(r + 4 * q);
                    for (int c = 1; c < nsplit; ++c) {
                        const float4 w = *reinterpret_cast<const float4 *>(r + c * split_stride + 4 * q);
                        v.x += w.x;
                        v.y += w.y;
                        v.z += w.z;
                        v.w += w.w;
                    }
                    // slots at or beyond m: zero (the G rows and columns there are zero)
                    rv[4 * q] = v.x;
                    rv[4 * q + 1] = 4 * q + 1 < m ? v.y : T(0);
                    rv[4 * q + 2] = 4 * q + 2 < m ? v.z : T(0);
                    rv[4 * q + 3] = 4 * q + 3 < m ? v.w : T(0);
                } else {
                    rv[4 * q] = rv[4 * q + 1] = rv[4 * q + 2] = rv[4 * q + 3] = T(0);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) {
                T rj = T(0);
                if (j < m) {
                    rj = r[j];
                    for (int c = 1; c < nsplit; ++c) rj += r[c * split_stride + j];
                }
                rv[j] = rj;
            }
        }
        const T *G = gram + (size_t)a * M * M;
        T ov[MS];
#pragma unroll
        for (int q = 0; q < MS; ++q) ov[q] = T(0);
#pragma unroll
        for (int q = 0; q < M; ++q) {
            T acc = T(0);
            if constexpr (V4 && M % 4 == 0) {
#pragma unroll
                for (int c = 0; c < M / 4; ++c) {
                    const float4 gq = __ldg(reinterpret_cast<const float4 *>(G + q * M) + c);
                    acc = fma(gq.x, rv[4 * c], acc);
                    acc = fma(gq.y, rv[4 * c + 1], acc);
                    acc = fma(gq.z, rv[4 * c + 2], acc);
                    acc = fma(gq.w, rv[4 * c + 3], acc);
                }
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j) acc = fma(__ldg(G + q * M + j), rv[j], acc);
            }
            ov[q] = acc;
        }
        T *dst = gt + i * MS;
        if constexpr (V4 && MS % 4 == 0) {
#pragma unroll
            for (int q = 0; q < MS / 4; ++q)
                reinterpret_cast<float4 *>(dst)[q] = make_float4(ov[4 * q], ov[4 * q + 1], ov[4 * q + 2], ov[4 * q + 3]);
        } else {
#pragma unroll
            for (int q = 0; q < MS; ++q) dst[q] = ov[q];
        }
    }
}

template <typename S, typename T, int M>
dr_status fold_normal_launch_t(dr_plan *P, const void *x, void *y, cudaStream_t st) {
    if (!P->d_fold_gram) return fail(DR_EINVAL, "folded normal operator unavailable for this plan");
    StaticOut rs{};
    {
        dr_status s = fold_static_dispatch<S, T, M>(P, x, st, rs);
        if (s != DR_OK) return s;
    }
    {
        dr_status s = ensure_fold_scratch(P);
        if (s != DR_OK) return s;
    }
    fold_gram_kernel<T, M><<<red_grid((size_t)P->nz * P->fold_U * P->ns), kRedThreads, 0, st>>>(
        (const T *)rs.ru, (T *)P->d_gt, (const T *)P->d_fold_gram, P->nz, P->fold_U, P->ns, rs.ms_ru, P->m, rs.nsplit,
        rs.split_stride);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fold_gram_kernel launch");
    return fold_backproject<S, T, M>(P, y, 1.0, 0.0, true, st);
}

template <typename S, typename T>
struct FoldOps {
    static dr_status fwd(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                         cudaStream_t st);
    static dr_status fwd2(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                          cudaStream_t st);
    static dr_status adj(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                         cudaStream_t st);
    // y = R*R x on compute-typed buffers (static transforms, Gram mix, back-projection)
    static dr_status normal(dr_plan *P, const void *x, void *y, cudaStream_t st);
};

#define DR_FOLD_DISPATCH(FN, S, T, ...)                   \
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
dr_status FoldOps<S, T>::fwd(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                             cudaStream_t st) {
    DR_FOLD_DISPATCH(fold_fwd_launch_t, S, T, P, u, out, gm, mode, sigma, st)
}

template <typename S, typename T>
dr_status FoldOps<S, T>::fwd2(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                              cudaStream_t st) {
    DR_FOLD_DISPATCH(fold_fwd2_launch_t, S, T, P, u, out, gm, mode, sigma, st)
}

template <typename S, typename T>
dr_status FoldOps<S, T>::adj(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                             cudaStream_t st) {
    DR_FOLD_DISPATCH(fold_adj_launch_t, S, T, P, g, u, alpha, beta, u_calc, st)
}

template <typename S, typename T>
dr_status FoldOps<S, T>::normal(dr_plan *P, const void *x, void *y, cudaStream_t st) {
    DR_FOLD_DISPATCH(fold_normal_launch_t, S, T, P, x, y, st)
}

extern template struct FoldOps<float, float>;
extern template struct FoldOps<bf16, float>;

}  // namespace dr
