// dr_device.cuh -- device helpers: storage conversions, block reductions with
// a deterministic last-block finish, and the mbarrier / TMA inline PTX used by
// the staged kernels.
#pragma once

#include "dr_internal.cuh"

namespace dr {

// Per-thread partial sum of a reduction whose total is accumulated in double
// across threads and blocks.  For float terms the thread's own sum is
// compensated (Kahan summation: the rounding error of every addition is
// carried in c and fed back), so its error stays at a few float roundings of
// the sum of magnitudes however many terms the thread adds, and the FP64 pipe
// is touched once per thread instead of once per term.  Double terms are
// added directly.
template <typename T>
struct PartialSum {
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T x) {
        if constexpr (sizeof(T) == 4) {
            const T y = x - c;
            const T t = s + y;
            c = (t - s) - y;
            s = t;
        } else {
            s += x;
        }
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Counter-based SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): output i of the
// stream with seed s is the finaliser applied to s + (i+1) * golden gamma.
__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// ---------------------------------------------------------------------------
// Storage <-> compute conversions
// ---------------------------------------------------------------------------
template <typename T, typename S>
__device__ __forceinline__ T ldc(const S *p);
template <>
__device__ __forceinline__ float ldc<float, float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float ldc<float, bf16>(const bf16 *p) { return __bfloat162float(*p); }
template <>
__device__ __forceinline__ double ldc<double, double>(const double *p) { return *p; }

template <typename T, typename S>
__device__ __forceinline__ void stc(S *p, T v);
template <>
__device__ __forceinline__ void stc<float, float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void stc<float, bf16>(bf16 *p, float v) { *p = __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ void stc<double, double>(double *p, double v) { *p = v; }

// Load m (<= M) consecutive coefficients; lanes j >= m are zero.
template <typename T, typename S, int M>
__device__ __forceinline__ void load_coeffs(const S *__restrict__ p, int m, T (&out)[M]) {
    if constexpr (sizeof(S) == 4 && (M % 4) == 0) {
        if (m == M) {
            const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
            for (int j = 0; j < M / 4; ++j) {
                const float4 v = __ldg(q + j);
                out[4 * j] = v.x;
                out[4 * j + 1] = v.y;
                out[4 * j + 2] = v.z;
                out[4 * j + 3] = v.w;
            }
            return;
        }
    }
    if constexpr (sizeof(S) == 2 && (M % 8) == 0) {
        if (m == M) {
            const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
            for (int j = 0; j < M / 8; ++j) {
                const uint4 v = __ldg(q + j);
                const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    out[8 * j + 2 * h] = __uint_as_float(w[h] << 16);
                    out[8 * j + 2 * h + 1] = __uint_as_float(w[h] & 0xffff0000u);
                }
            }
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < M; ++j) out[j] = (j < m) ? ldc<T>(p + j) : T(0);
}

// Compute-typed rows of m (<= M) values that the calling kernel also writes:
// plain (coherent) loads, and stores of the first m values; 16-byte vectors
// when the row is a whole number of them.
template <typename T, int M>
__device__ __forceinline__ void load_row(const T *p, int m, T (&out)[M]) {
    if constexpr (sizeof(T) == 4 && (M % 4) == 0) {
        if (m == M) {
#pragma unroll
            for (int j = 0; j < M / 4; ++j) {
                const float4 v = reinterpret_cast<const float4 *>(p)[j];
                out[4 * j] = v.x;
                out[4 * j + 1] = v.y;
                out[4 * j + 2] = v.z;
                out[4 * j + 3] = v.w;
            }
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < M; ++j) out[j] = (j < m) ? p[j] : T(0);
}

template <typename T, int M>
__device__ __forceinline__ void store_row(T *p, int m, const T (&v)[M]) {
    if constexpr (sizeof(T) == 4 && (M % 4) == 0) {
        if (m == M) {
#pragma unroll
            for (int j = 0; j < M / 4; ++j)
                reinterpret_cast<float4 *>(p)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < M; ++j)
        if (j < m) p[j] = v[j];
}

// ---------------------------------------------------------------------------
// Reductions.  Each block reduces NV doubles, writes them to its partial
// slot, and the last block to finish sums all partials in a fixed order, so
// the result does not depend on block scheduling.  Returns true in thread 0
// of the last block, with the totals in `tot`.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ bool block_reduce_last(double (&v)[NV], double *__restrict__ partials,
                                                  unsigned *__restrict__ counter, double (&tot)[NV]) {
    __shared__ double sh[NV][32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int off = 16; off; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
        if (lane == 0) sh[k][warp] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[k][w];
            partials[(size_t)k * gridDim.x + blockIdx.x] = s;
        }
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    // last block: warp 0 sums the partials, lane-strided then a fixed tree
    __threadfence();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int b = lane; b < (int)gridDim.x; b += 32)
                s += __ldcg(partials + (size_t)k * gridDim.x + b);
#pragma unroll
            for (int off = 16; off; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            tot[k] = s;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
    return threadIdx.x == 0;
}

// ---------------------------------------------------------------------------
// mbarrier + TMA (inline PTX, sm_90+ / sm_100 family).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier, giving up after `limit_ns`
// nanoseconds of wall time; on give-up sets the status bit and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, int *status,
                                                  unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0u && global_ns() - t0 > limit_ns) {
            atomicOr(status, kStatusTimeout);
            return false;
        }
    }
}

// As mbar_wait_bounded, but also gives up as soon as another CTA has set the
// status word (a pipeline that stalls everywhere then ends within one limit).
__device__ __forceinline__ bool mbar_wait_bounded_any(uint64_t *bar, unsigned parity, int *status,
                                                      unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0u) {
            if (*(volatile int *)status != 0) return false;
            if (global_ns() - t0 > limit_ns) {
                atomicOr(status, kStatusTimeout);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Ampere-style asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async_16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace dr
