// solver.cu -- iterative solvers for the model of Eq. (lr12) on the device:
// ADMM with a conjugate-gradient u-step, and Chambolle-Pock (Sec. 3, Fig. 2).
//
// All inner products, CG step sizes and residuals are accumulated in double
// on the device (deterministic last-block reductions) and never leave it
// inside an iteration, so one iteration is a fixed launch sequence that is
// captured once as a CUDA graph and replayed.  A device-side iteration
// counter tells the reducing kernels which objective row to write.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "dr_device.cuh"

namespace dr {

// 16-byte vectors of the compute type: the vector kernels below move whole
// vectors when every pointer they touch is 16-byte aligned (VEC), else single
// elements.  Products are formed in the compute type, each thread sums its
// own terms in a compensated PartialSum, and the thread totals are
// accumulated in double across the block and the grid, in a fixed order
// (deterministic for a given n and grid).  Double arithmetic per element
// would dominate these kernels: FP64 runs at a small fraction of the FP32 rate
// on this GPU.
template <typename T>
struct V16;
template <>
struct V16<float> {
    using type = float4;
    static constexpr int W = 4;
    __device__ static float get(const float4 &v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)); }
    __device__ static void set(float4 &v, int k, float x) {
        if (k == 0) v.x = x;
        else if (k == 1) v.y = x;
        else if (k == 2) v.z = x;
        else v.w = x;
    }
};
template <>
struct V16<double> {
    using type = double2;
    static constexpr int W = 2;
    __device__ static double get(const double2 &v, int k) { return k == 0 ? v.x : v.y; }
    __device__ static void set(double2 &v, int k, double x) {
        if (k == 0) v.x = x;
        else v.y = x;
    }
};

inline bool aligned16(const void *a, const void *b = nullptr, const void *c = nullptr, const void *d = nullptr) {
    return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d) & 15u) == 0;
}

template <typename T, bool VEC>
__global__ void __launch_bounds__(kRedThreads)
    dot_kernel(const T *__restrict__ a, const T *__restrict__ b, size_t n, double *partials, unsigned *counter,
               DevScalars *scal, double *obj, int row_off, int col, int to_lam) {
    PartialSum<T> acc;
    const size_t stride = (size_t)gridDim.x * blockDim.x, tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t done = 0;
    if constexpr (VEC) {
        using V = V16<T>;
        const size_t nv = n / V::W;
        const typename V::type *av = reinterpret_cast<const typename V::type *>(a);
        const typename V::type *bv = reinterpret_cast<const typename V::type *>(b);
        for (size_t i = tid; i < nv; i += stride) {
            const typename V::type x = __ldg(av + i), y = __ldg(bv + i);
            T s = T(0);
#pragma unroll
            for (int k = 0; k < V::W; ++k) s = fma(V::get(x, k), V::get(y, k), s);
            acc.add(s);
        }
        done = nv * V::W;
    }
    for (size_t i = done + tid; i < n; i += stride) acc.add(a[i] * b[i]);
    double v[1] = {acc.value()}, tot[1];
    if (block_reduce_last<1>(v, partials, counter, tot)) {
        if (obj) obj[3 * (size_t)(scal->iter + row_off) + col] = tot[0];
        if (to_lam) scal->lam = tot[0];
        if (!obj && !to_lam) scal->acc0 = tot[0];
    }
}

// u += alpha p; r -= alpha q; rr_new = <r, r>; beta = rr_new / rr.
template <typename T, bool VEC>
__global__ void __launch_bounds__(kRedThreads)
    cg_update_kernel(T *__restrict__ u, T *__restrict__ r, const T *__restrict__ p, const T *__restrict__ q,
                     size_t n, double *partials, unsigned *counter, DevScalars *scal) {
    const T a = (T)scal->alpha;
    PartialSum<T> acc;
    const size_t stride = (size_t)gridDim.x * blockDim.x, tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t done = 0;
    if constexpr (VEC) {
        using V = V16<T>;
        using VT = typename V::type;
        const size_t nv = n / V::W;
        VT *uv = reinterpret_cast<VT *>(u), *rv = reinterpret_cast<VT *>(r);
        const VT *pv = reinterpret_cast<const VT *>(p), *qv = reinterpret_cast<const VT *>(q);
        for (size_t i = tid; i < nv; i += stride) {
            VT uu = uv[i], rr = rv[i];
            const VT pp = __ldg(pv + i), qq = __ldg(qv + i);
            T s = T(0);
#pragma unroll
            for (int k = 0; k < V::W; ++k) {
                V::set(uu, k, V::get(uu, k) + a * V::get(pp, k));
                const T rn = V::get(rr, k) - a * V::get(qq, k);
                V::set(rr, k, rn);
                s = fma(rn, rn, s);
            }
            acc.add(s);
            uv[i] = uu;
            rv[i] = rr;
        }
        done = nv * V::W;
    }
    for (size_t i = done + tid; i < n; i += stride) {
        u[i] += a * p[i];
        const T rn = r[i] - a * q[i];
        r[i] = rn;
        acc.add(rn * rn);
    }
    double v[1] = {acc.value()}, tot[1];
    if (block_reduce_last<1>(v, partials, counter, tot)) {
        if (scal->active) {
            scal->beta = tot[0] / scal->rr;
            scal->rr = tot[0];
        } else {
            scal->beta = 0.0;
        }
    }
}

template <typename T, bool VEC>
__global__ void cg_dir_kernel(T *__restrict__ p, const T *__restrict__ r, size_t n, const DevScalars *scal) {
    const T b = (T)scal->beta;
    const size_t stride = (size_t)gridDim.x * blockDim.x, tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t done = 0;
    if constexpr (VEC) {
        using V = V16<T>;
        using VT = typename V::type;
        const size_t nv = n / V::W;
        VT *pv = reinterpret_cast<VT *>(p);
        const VT *rv = reinterpret_cast<const VT *>(r);
        for (size_t i = tid; i < nv; i += stride) {
            VT pp = pv[i];
            const VT rr = __ldg(rv + i);
#pragma unroll
            for (int k = 0; k < V::W; ++k) V::set(pp, k, V::get(rr, k) + b * V::get(pp, k));
            pv[i] = pp;
        }
        done = nv * V::W;
    }
    for (size_t i = done + tid; i < n; i += stride) p[i] = r[i] + b * p[i];
}

// Power-iteration start x_i = 0.5 + U_i (SplitMix64 stream, seed 1809) for
// global indices i = first .. first + n - 1.
template <typename T>
__global__ void pow_init_kernel(T *__restrict__ x, size_t n, size_t first) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = (T)(0.5 + splitmix_uniform(1809ull, (unsigned long long)(first + i)));
}

// x = y / sqrt(scal->lam) (normalise by the norm just reduced).
template <typename T>
__global__ void pow_scale_kernel(T *__restrict__ x, const T *__restrict__ y, size_t n, const DevScalars *scal) {
    const double nrm = sqrt(scal->lam);
    const T f = nrm > 0.0 ? (T)(1.0 / nrm) : T(0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = y[i] * f;
}

__global__ void iter_kernel(DevScalars *scal, int set, int value) {
    if (set) scal->iter = value;
    else scal->iter += 1;
}

template <typename S, typename T>
__global__ void convert_kernel(const S *__restrict__ in, T *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        stc<T>(out + i, ldc<T>(in + i));
}
template <>
__global__ void convert_kernel<float, bf16>(const float *__restrict__ in, bf16 *__restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

static dr_status launched(const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DR_OK : cuda_fail(e, what);
}

static int vec_grid(size_t n) { return red_grid(n); }

// ---------------------------------------------------------------------------
// typed launch helpers (T = float or double)
// ---------------------------------------------------------------------------
template <typename T>
static dr_status dot_t(dr_plan *P, const void *a, const void *b, size_t n, int slot, double *obj, int row_off,
                       int col, int to_lam, cudaStream_t st) {
    if (aligned16(a, b))
        dot_kernel<T, true><<<vec_grid(n), kRedThreads, 0, st>>>((const T *)a, (const T *)b, n,
                                                                 P->d_partials + slot * kRedSlotStride,
                                                                 P->d_counters + slot, P->d_scal, obj, row_off, col,
                                                                 to_lam);
    else
        dot_kernel<T, false><<<vec_grid(n), kRedThreads, 0, st>>>((const T *)a, (const T *)b, n,
                                                                  P->d_partials + slot * kRedSlotStride,
                                                                  P->d_counters + slot, P->d_scal, obj, row_off, col,
                                                                  to_lam);
    return launched("dot_kernel");
}

dr_status launch_dot_to(dr_plan *P, const void *a, const void *b, size_t n, bool storage, double *dst,
                        cudaStream_t st) {
    (void)storage;
    (void)dst;
    if (P->prec == DR_F64) return dot_t<double>(P, a, b, n, kSlotDot, nullptr, 0, 0, 0, st);
    return dot_t<float>(P, a, b, n, kSlotDot, nullptr, 0, 0, 0, st);
}

void free_workspace(dr_plan *P) {
    Workspace &w = P->ws;
    void *ptrs[] = {w.r, w.p, w.q, w.ut, w.uold, w.gd, w.h1, w.mu, w.w, w.u_dev, w.g_dev, w.obj};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    w = Workspace();
}

static size_t ws_bytes(const dr_plan *P, dr_algo algo, int iters) {
    const size_t T = calc_size(P->prec), F = field_size(P);
    const size_t nu = nu_elems(P), ng = ng_elems(P), nf = nf_elems(P);
    size_t b = 0;
    if (algo == DR_ADMM_CG) b += 3 * nu * T + ng * T + 2 * nf * F;
    else b += 2 * nu * T + 2 * ng * T + nf * F;
    b += nu * T + ng * T;  // internal copies of u and g (host or bf16 inputs)
    b += sizeof(double) * 3 * (size_t)(iters + 1);
    return b;
}

static dr_status ensure_ws(dr_plan *P, dr_algo algo, int iters) {
    Workspace &w = P->ws;
    if (w.bytes && w.algo == algo && w.obj_cap >= iters + 1) return DR_OK;
    free_workspace(P);
    const size_t T = calc_size(P->prec), F = field_size(P);
    const size_t nu = nu_elems(P), ng = ng_elems(P), nf = nf_elems(P);
    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
        w.bytes += bytes;
        return true;
    };
    bool ok = true;
    if (algo == DR_ADMM_CG) {
        ok = ok && alloc(&w.r, nu * T) && alloc(&w.p, nu * T) && alloc(&w.q, nu * T);
        ok = ok && alloc(&w.gd, ng * T) && alloc(&w.mu, nf * F) && alloc(&w.w, nf * F);
    } else {
        ok = ok && alloc(&w.ut, nu * T) && alloc(&w.q, nu * T);
        ok = ok && alloc(&w.gd, ng * T) && alloc(&w.h1, ng * T) && alloc(&w.mu, nf * F);
    }
    ok = ok && alloc(&w.u_dev, nu * T) && alloc(&w.g_dev, ng * T);
    ok = ok && alloc((void **)&w.obj, sizeof(double) * 3 * (size_t)(iters + 1));
    if (!ok) {
        cudaGetLastError();
        free_workspace(P);
        return fail(DR_ENOMEM, "admm_solve: device workspace allocation failed");
    }
    w.algo = algo;
    w.obj_cap = iters + 1;
    return DR_OK;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
static dr_status vec_launches(dr_plan *P, int which, void *a, void *b, void *c, void *d, size_t n, cudaStream_t st) {
    switch (which) {
        case 0:
            if (aligned16(a, b, c, d))
                cg_update_kernel<T, true><<<vec_grid(n), kRedThreads, 0, st>>>(
                    (T *)a, (T *)b, (const T *)c, (const T *)d, n, P->d_partials + kSlotUpd * kRedSlotStride,
                    P->d_counters + kSlotUpd, P->d_scal);
            else
                cg_update_kernel<T, false><<<vec_grid(n), kRedThreads, 0, st>>>(
                    (T *)a, (T *)b, (const T *)c, (const T *)d, n, P->d_partials + kSlotUpd * kRedSlotStride,
                    P->d_counters + kSlotUpd, P->d_scal);
            return launched("cg_update_kernel");
        case 1:
            if (aligned16(a, b))
                cg_dir_kernel<T, true><<<vec_grid(n), kRedThreads, 0, st>>>((T *)a, (const T *)b, n, P->d_scal);
            else
                cg_dir_kernel<T, false><<<vec_grid(n), kRedThreads, 0, st>>>((T *)a, (const T *)b, n, P->d_scal);
            return launched("cg_dir_kernel");
        case 2:
            pow_init_kernel<T><<<vec_grid(n), kRedThreads, 0, st>>>((T *)a, n, (size_t)0);
            return launched("pow_init_kernel");
        case 3:
            pow_scale_kernel<T><<<vec_grid(n), kRedThreads, 0, st>>>((T *)a, (const T *)b, n, P->d_scal);
            return launched("pow_scale_kernel");
    }
    return fail(DR_EINVAL, "vec_launches");
}

static dr_status vec(dr_plan *P, int which, void *a, void *b, void *c, void *d, size_t n, cudaStream_t st) {
    return P->prec == DR_F64 ? vec_launches<double>(P, which, a, b, c, d, n, st)
                             : vec_launches<float>(P, which, a, b, c, d, n, st);
}

static dr_status dot(dr_plan *P, const void *a, const void *b, size_t n, int slot, double *obj, int row_off, int col,
                     int to_lam, cudaStream_t st) {
    return P->prec == DR_F64 ? dot_t<double>(P, a, b, n, slot, obj, row_off, col, to_lam, st)
                             : dot_t<float>(P, a, b, n, slot, obj, row_off, col, to_lam, st);
}

// Helpers for the slab-streamed solver (slabs.cu).
dr_status launch_dot_obj(dr_plan *P, const void *a, const void *b, size_t n, double *obj, int row_off, int col,
                         cudaStream_t st) {
    return dot(P, a, b, n, kSlotFid, obj, row_off, col, 0, st);
}

dr_status launch_set_iter(dr_plan *P, int value, cudaStream_t st) {
    iter_kernel<<<1, 1, 0, st>>>(P->d_scal, 1, value);
    return launched("iter_kernel");
}

dr_status launch_pow_init(dr_plan *P, void *x, size_t n, size_t first, cudaStream_t st) {
    if (P->prec == DR_F64) pow_init_kernel<double><<<vec_grid(n), kRedThreads, 0, st>>>((double *)x, n, first);
    else pow_init_kernel<float><<<vec_grid(n), kRedThreads, 0, st>>>((float *)x, n, first);
    return launched("pow_init_kernel");
}

dr_status launch_convert_bf16(dr_plan *P, const void *in, void *out, size_t n, bool to_bf16, cudaStream_t st) {
    (void)P;
    if (to_bf16) convert_kernel<float, bf16><<<vec_grid(n), kRedThreads, 0, st>>>((const float *)in, (bf16 *)out, n);
    else convert_kernel<bf16, float><<<vec_grid(n), kRedThreads, 0, st>>>((const bf16 *)in, (float *)out, n);
    return launched("convert_kernel");
}

#define TRY(...)                       \
    do {                               \
        dr_status _s = (__VA_ARGS__);  \
        if (_s != DR_OK) return _s;    \
    } while (0)

// The projector/TV launchers take "calc" (compute-typed) buffers here.
dr_status launch_fwd_calc(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                          cudaStream_t st);
dr_status launch_adj_calc(dr_plan *P, const void *g, void *u, double alpha, double beta, cudaStream_t st);

// One ADMM-CG iteration (the captured sequence).
static dr_status admm_iteration(dr_plan *P, void *u, const void *g, const dr_solve_params &prm, double rho,
                                cudaStream_t st) {
    Workspace &w = P->ws;
    const size_t nu = nu_elems(P), ng = ng_elems(P);
    // d = R u - g ; fidelity of the current u ; r = R*(g - R u)
    TRY(launch_fwd_calc(P, u, w.gd, g, 1, 0.0, st));
    TRY(dot(P, w.gd, w.gd, ng, kSlotFid, w.obj, 0, 0, 0, st));
    TRY(launch_adj_calc(P, w.gd, w.r, -1.0, 0.0, st));
    // r += rho (D^T w - D^T D u); p = r; rr = <r,r>
    TRY(launch_rhs(P, u, w.w, w.r, w.p, rho, prm.lambda2, st));
    for (int c = 0; c < prm.n_cg; ++c) {
        TRY(launch_normal_calc(P, w.p, w.q, w.gd, st));  // q = R*R p
        TRY(launch_lap(P, w.p, w.q, rho, 1.0, prm.lambda2, 1, st));
        TRY(vec(P, 0, u, w.r, w.p, w.q, nu, st));
        if (c + 1 < prm.n_cg) TRY(vec(P, 1, w.p, w.r, nullptr, nullptr, nu, st));
    }
    TRY(launch_prox(P, u, true, w.mu, w.w, rho, prm.lambda1, prm.lambda2, w.obj + 3, st));
    iter_kernel<<<1, 1, 0, st>>>(P->d_scal, 0, 0);
    return launched("iter_kernel");
}

static dr_status cp_iteration(dr_plan *P, void *u, const void *g, const dr_solve_params &prm, double sigma,
                              double tau, bool want_obj, cudaStream_t st) {
    Workspace &w = P->ws;
    const size_t ng = ng_elems(P);
    TRY(launch_fwd_calc(P, w.ut, w.h1, g, 2, sigma, st));
    TRY(launch_cp_dual(P, w.ut, w.mu, sigma, prm.lambda1, prm.lambda2, st));
    TRY(launch_adj_calc(P, w.h1, w.q, 1.0, 0.0, st));
    TRY(launch_cp_primal(P, u, w.ut, w.q, w.mu, tau, prm.cp_theta, prm.lambda2, st));
    if (want_obj) {
        TRY(launch_fwd_calc(P, u, w.gd, g, 1, 0.0, st));
        TRY(dot(P, w.gd, w.gd, ng, kSlotFid, w.obj, 1, 0, 0, st));
        TRY(launch_tv_sum(P, u, prm.lambda2, w.obj + 3, st));
    }
    iter_kernel<<<1, 1, 0, st>>>(P->d_scal, 0, 0);
    return launched("iter_kernel");
}

static dr_status power_norm(dr_plan *P, double lambda2, int iters, double *L, cudaStream_t st) {
    Workspace &w = P->ws;
    const size_t nu = nu_elems(P);
    void *x = w.ut, *y = w.q;
    TRY(vec(P, 2, x, nullptr, nullptr, nullptr, nu, st));
    TRY(dot(P, x, x, nu, kSlotPow, nullptr, 0, 0, 1, st));
    TRY(vec(P, 3, x, x, nullptr, nullptr, nu, st));
    for (int it = 0; it < iters; ++it) {
        TRY(launch_normal_calc(P, x, y, w.gd, st));  // y = R*R x
        TRY(launch_lap(P, x, y, 1.0, 1.0, lambda2, 0, st));
        TRY(dot(P, y, y, nu, kSlotPow, nullptr, 0, 0, 1, st));
        TRY(vec(P, 3, x, y, nullptr, nullptr, nu, st));
    }
    DevScalars hs;
    cudaError_t e = cudaMemcpyAsync(&hs, P->d_scal, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "power_norm: read");
    *L = std::sqrt(std::sqrt(hs.lam));
    return DR_OK;
}

template <typename S, typename T>
static dr_status convert(const void *in, void *out, size_t n, cudaStream_t st) {
    convert_kernel<S, T><<<vec_grid(n), kRedThreads, 0, st>>>((const S *)in, (T *)out, n);
    return launched("convert_kernel");
}

// Per-call solver state: which device buffers hold g and u, step sizes.
struct SolveCtx {
    dr_solve_params prm;
    const void *g_in = nullptr;
    void *u_io = nullptr;
    const void *g = nullptr;  // compute-typed device copy or the caller's buffer
    void *u = nullptr;
    bool g_dev = false, u_dev = false, bf = false, want_obj = false;
    double rho = 0.0, sigma = 0.0, tau = 0.0, L = 0.0;
    int done = 0;             // iterations issued
};

// Stage inputs, reset the state, run the Chambolle-Pock power iteration.
static dr_status solve_begin(dr_plan *P, const void *g_in, void *u_io, const dr_solve_params &prm, SolveCtx &c) {
    const cudaStream_t st = P->graph_stream;
    Workspace &w = P->ws;
    const size_t nu = nu_elems(P), ng = ng_elems(P), nf = nf_elems(P);
    const size_t es = elem_size(P->prec), cs = calc_size(P->prec);
    c.prm = prm;
    c.g_in = g_in;
    c.u_io = u_io;
    c.bf = P->prec == DR_BF16_F32ACC;
    c.g_dev = is_device_ptr(g_in);
    c.u_dev = is_device_ptr(u_io);
    c.want_obj = prm.objective_out != nullptr;
    c.done = 0;

    DR_CUDA_TRY(cudaEventRecord(P->ev_a, P->stream));
    DR_CUDA_TRY(cudaStreamWaitEvent(st, P->ev_a, 0));
    // pick the faster projector variants once per plan (scratch: q, gd)
    if (!P->tuned && (P->var_fwd < 0 || P->var_adj < 0)) TRY(autotune(P, w.q, w.gd));

    // ---- bring g and u into compute-typed device buffers ----
    c.g = g_in;
    c.u = u_io;
    if (!c.g_dev || c.bf) {
        void *src = (void *)g_in;
        if (!c.g_dev) {
            // host data: copy raw storage-typed bytes, then convert if needed
            void *stage = c.bf ? w.gd : w.g_dev;  // gd is large enough (ng * cs >= ng * es)
            DR_CUDA_TRY(cudaMemcpyAsync(stage, g_in, ng * es, cudaMemcpyHostToDevice, st));
            src = stage;
        }
        if (c.bf) TRY(convert<bf16, float>(src, w.g_dev, ng, st));
        c.g = w.g_dev;
    }
    if (!c.u_dev || c.bf) {
        void *src = u_io;
        if (!c.u_dev) {
            void *stage = c.bf ? w.q : w.u_dev;
            DR_CUDA_TRY(cudaMemcpyAsync(stage, u_io, nu * es, cudaMemcpyHostToDevice, st));
            src = stage;
        }
        if (c.bf) TRY(convert<bf16, float>(src, w.u_dev, nu, st));
        c.u = w.u_dev;
    }

    DR_CUDA_TRY(cudaMemsetAsync(P->d_scal, 0, sizeof(DevScalars), st));
    DR_CUDA_TRY(cudaMemsetAsync(w.obj, 0, sizeof(double) * 3 * (size_t)(prm.iters + 1), st));
    c.rho = prm.rho > 0.0 ? prm.rho : (prm.lambda1 > 0.0 ? 10.0 * prm.lambda1 : 1.0);

    // the state besides u: zero at a fresh start, the caller's on resume
    const unsigned char *rs = prm.resume ? (const unsigned char *)prm.state : nullptr;
    const size_t fsz = nf * field_size(P);  // bytes of one dual field
    if (prm.algo == DR_ADMM_CG) {
        if (rs) {
            DR_CUDA_TRY(cudaMemcpyAsync(w.mu, rs, fsz, cudaMemcpyDeviceToDevice, st));
            DR_CUDA_TRY(cudaMemcpyAsync(w.w, rs + fsz, fsz, cudaMemcpyDeviceToDevice, st));
        } else {
            DR_CUDA_TRY(cudaMemsetAsync(w.mu, 0, fsz, st));
            DR_CUDA_TRY(cudaMemsetAsync(w.w, 0, fsz, st));
        }
    } else {
        if (rs) {
            DR_CUDA_TRY(cudaMemcpyAsync(w.mu, rs, fsz, cudaMemcpyDeviceToDevice, st));
            DR_CUDA_TRY(cudaMemcpyAsync(w.h1, rs + fsz, ng * cs, cudaMemcpyDeviceToDevice, st));
        } else {
            DR_CUDA_TRY(cudaMemsetAsync(w.h1, 0, ng * cs, st));
            DR_CUDA_TRY(cudaMemsetAsync(w.mu, 0, fsz, st));
        }
        if (prm.op_norm > 0.0) {
            c.L = prm.op_norm;
        } else {
            const int pit = prm.power_iters > 0 ? prm.power_iters : 100;
            TRY(power_norm(P, prm.lambda2, pit, &c.L, st));
        }
        if (!(c.L > 0.0) || !std::isfinite(c.L)) return fail(DR_EINVAL, "admm_solve: operator norm is zero");
        c.sigma = c.tau = 0.99 / c.L;
        if (prm.op_norm_out) *prm.op_norm_out = c.L;
        DR_CUDA_TRY(cudaMemcpyAsync(w.ut, rs ? (const void *)(rs + (nf + ng) * cs) : (const void *)c.u, nu * cs,
                                    cudaMemcpyDeviceToDevice, st));
        iter_kernel<<<1, 1, 0, st>>>(P->d_scal, 1, 0);
        TRY(launched("iter_kernel"));
    }
    return DR_OK;
}

// Launch one iteration of the chosen algorithm on stream s.
static dr_status solve_iter(dr_plan *P, SolveCtx &c, cudaStream_t s) {
    if (c.prm.algo == DR_ADMM_CG) return admm_iteration(P, c.u, c.g, c.prm, c.rho, s);
    return cp_iteration(P, c.u, c.g, c.prm, c.sigma, c.tau, c.want_obj, s);
}

// Final objective row, results back to the caller's buffers, status check.
static dr_status solve_end(dr_plan *P, SolveCtx &c) {
    const cudaStream_t st = P->graph_stream;
    Workspace &w = P->ws;
    const dr_solve_params &prm = c.prm;
    const size_t nu = nu_elems(P), ng = ng_elems(P);
    const size_t es = elem_size(P->prec), cs = calc_size(P->prec);
    if (prm.iters > 0 && prm.algo == DR_ADMM_CG && c.want_obj) {
        // fidelity of the final u (row iters)
        TRY(launch_fwd_calc(P, c.u, w.gd, c.g, 1, 0.0, st));
        TRY(dot(P, w.gd, w.gd, ng, kSlotFid, w.obj, 0, 0, 0, st));
    }
    if (prm.state) {
        // the state besides u, for a later call to continue from
        unsigned char *sd = (unsigned char *)prm.state;
        const size_t fsz = nf_elems(P) * field_size(P);
        if (prm.algo == DR_ADMM_CG) {
            DR_CUDA_TRY(cudaMemcpyAsync(sd, w.mu, fsz, cudaMemcpyDeviceToDevice, st));
            DR_CUDA_TRY(cudaMemcpyAsync(sd + fsz, w.w, fsz, cudaMemcpyDeviceToDevice, st));
        } else {
            DR_CUDA_TRY(cudaMemcpyAsync(sd, w.mu, fsz, cudaMemcpyDeviceToDevice, st));
            DR_CUDA_TRY(cudaMemcpyAsync(sd + fsz, w.h1, ng * cs, cudaMemcpyDeviceToDevice, st));
            DR_CUDA_TRY(cudaMemcpyAsync(sd + fsz + ng * cs, w.ut, nu * cs, cudaMemcpyDeviceToDevice, st));
        }
    }
    if (!c.u_dev || c.bf) {
        void *dst = c.u_io;
        if (c.bf) {
            void *tmp = c.u_dev ? c.u_io : (void *)w.q;
            TRY(convert<float, bf16>(c.u, tmp, nu, st));
            if (!c.u_dev) DR_CUDA_TRY(cudaMemcpyAsync(dst, tmp, nu * es, cudaMemcpyDeviceToHost, st));
        } else {
            DR_CUDA_TRY(cudaMemcpyAsync(dst, c.u, nu * cs, cudaMemcpyDeviceToHost, st));
        }
    }
    std::vector<double> obj;
    if (prm.iters > 0 && (c.want_obj || prm.primal_res_out)) {
        obj.resize(3 * (size_t)(prm.iters + 1));
        DR_CUDA_TRY(cudaMemcpyAsync(obj.data(), w.obj, sizeof(double) * obj.size(), cudaMemcpyDeviceToHost, st));
    }
    DevScalars hs;
    DR_CUDA_TRY(cudaMemcpyAsync(&hs, P->d_scal, sizeof(hs), cudaMemcpyDeviceToHost, st));
    DR_CUDA_TRY(cudaEventRecord(P->ev_b, st));
    DR_CUDA_TRY(cudaStreamWaitEvent(P->stream, P->ev_b, 0));
    DR_CUDA_TRY(cudaStreamSynchronize(st));
    int flag = 0;
    DR_CUDA_TRY(cudaMemcpy(&flag, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(P->d_status, 0, sizeof(int));
        return fail(DR_ETIMEOUT, "admm_solve: a bounded device-side wait gave up");
    }
    bool finite = std::isfinite(hs.rr) && std::isfinite(hs.alpha) && std::isfinite(hs.beta);
    for (int it = 0; it < prm.iters && !obj.empty(); ++it) {
        const double *row = &obj[3 * (size_t)(it + 1)];
        if (c.want_obj) prm.objective_out[it] = 0.5 * row[0] + prm.lambda1 * row[1];
        if (prm.primal_res_out) prm.primal_res_out[it] = std::sqrt(row[2]);
        if (c.want_obj && !std::isfinite(prm.objective_out[it])) finite = false;
    }
    if (!finite) return fail(DR_ENOTCONV, "admm_solve: non-finite values (check the data for NaN/Inf)");
    return DR_OK;
}

// Capture `body` (launches on per-job streams) as one graph on stream `root`.
// A device-wide call from another thread (a plan or buffer freed by another
// job) can invalidate a capture in progress; the capture is then repeated, a
// bounded number of times (the iteration bodies keep all state in device
// memory, so a discarded capture leaves nothing behind).
template <typename F>
static dr_status capture_graph(cudaStream_t root, F body, cudaGraphExec_t *exec) {
    dr_status last = DR_OK;
    for (int attempt = 0; attempt < 4; ++attempt) {
        cudaGraph_t graph = nullptr;
        DR_CUDA_TRY(cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal));
        const dr_status st = body();
        cudaError_t ce = cudaStreamEndCapture(root, &graph);
        if (st == DR_OK && ce == cudaSuccess) {
            ce = cudaGraphInstantiate(exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_fail(ce, "graph instantiate");
            return DR_OK;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();  // capture errors are not sticky
        last = st != DR_OK ? st : cuda_fail(ce, "graph capture");
        if (ce != cudaErrorStreamCaptureInvalidated) break;
    }
    return last;
}

// Cancellation of a serving job (P->cancel set): the host keeps at most two
// iterations in flight and looks at the flag before issuing the next one, so
// a raised flag stops the solve within about two iterations.  Returns true
// when the solve is to stop.
struct CancelGate {
    dr_plan *P;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    explicit CancelGate(dr_plan *p) : P(p) {
        if (P->cancel)
            for (auto &e : ev)
                if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) e = nullptr;
    }
    ~CancelGate() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    // before issuing iteration `it` (>= 1) on stream s
    bool stop(int it, cudaStream_t s) {
        if (!P->cancel) return false;
        if (it >= 3 && ev[it & 1]) cudaEventSynchronize(ev[it & 1]);  // iteration it - 2 has finished
        if (P->cancel->load(std::memory_order_relaxed)) {
            cudaStreamSynchronize(s);
            return true;
        }
        return false;
    }
    // after issuing iteration `it` on stream s
    void issued(int it, cudaStream_t s) {
        if (P->cancel && ev[it & 1]) cudaEventRecord(ev[it & 1], s);
    }
};

static dr_status solve(dr_plan *P, const void *g_in, void *u_io, const dr_solve_params &prm) {
    SolveCtx c;
    TRY(solve_begin(P, g_in, u_io, prm, c));
    const cudaStream_t st = P->graph_stream;
    CancelGate gate(P);
    if (prm.iters > 0) {
        // first iteration eagerly (sets kernel attributes, allocates lazily), the rest as one graph
        TRY(solve_iter(P, c, st));
        if (prm.iters > 1) {
            cudaGraphExec_t exec = nullptr;
            bool canceled = false;
            if (capture_graph(st, [&]() { return solve_iter(P, c, st); }, &exec) == DR_OK) {
                cudaError_t ce = cudaSuccess;
                for (int it = 1; it < prm.iters && ce == cudaSuccess; ++it) {
                    if (gate.stop(it, st)) {
                        canceled = true;
                        break;
                    }
                    ce = cudaGraphLaunch(exec, st);
                    gate.issued(it, st);
                }
                cudaGraphExecDestroy(exec);
                if (ce != cudaSuccess) return cuda_fail(ce, "admm_solve: graph launch");
            } else {
                // no graph: the same launches, issued one iteration at a time
                clear_error();
                for (int it = 1; it < prm.iters; ++it) {
                    if (gate.stop(it, st)) {
                        canceled = true;
                        break;
                    }
                    TRY(solve_iter(P, c, st));
                    gate.issued(it, st);
                }
            }
            if (canceled) {
                DR_CUDA_TRY(cudaStreamSynchronize(st));
                return fail(DR_ECANCELED, "admm_solve: canceled while running");
            }
        }
    }
    return solve_end(P, c);
}

// Several independent reconstructions: each iteration of all active jobs is
// one CUDA graph with one branch per job (fork from a root stream, join back),
// so the jobs' kernels overlap on the device.  Every job keeps its own plan,
// workspace, scalars and reduction slots, so its result is the same as alone.
static dr_status solve_batch(int n, dr_plan *const *plans, const void *const *g, void *const *u,
                             const dr_solve_params *prm) {
    std::vector<SolveCtx> c(n);
    for (int j = 0; j < n; ++j) TRY(solve_begin(plans[j], g[j], u[j], prm[j], c[j]));
    for (int j = 0; j < n; ++j)
        if (prm[j].iters > 0) {
            TRY(solve_iter(plans[j], c[j], plans[j]->graph_stream));
            c[j].done = 1;
        }
    cudaStream_t root = nullptr;
    DR_CUDA_TRY(cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking));
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    dr_status result = DR_OK;
    for (auto &e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) result = fail(DR_ECUDA, "batch events");
    // the root stream starts after every job's eager iteration
    for (int j = 0; j < n && result == DR_OK; ++j) {
        if (cudaEventRecord(ev[j + 1], plans[j]->graph_stream) != cudaSuccess ||
            cudaStreamWaitEvent(root, ev[j + 1], 0) != cudaSuccess)
            result = fail(DR_ECUDA, "batch: join eager iterations");
    }
    while (result == DR_OK) {
        std::vector<int> act;
        int reps = 1 << 30;
        for (int j = 0; j < n; ++j)
            if (c[j].done < prm[j].iters) {
                act.push_back(j);
                reps = std::min(reps, prm[j].iters - c[j].done);
            }
        if (act.empty()) break;
        cudaGraphExec_t exec = nullptr;
        result = capture_graph(
            root,
            [&]() -> dr_status {
                DR_CUDA_TRY(cudaEventRecord(ev[0], root));
                for (int j : act) {
                    DR_CUDA_TRY(cudaStreamWaitEvent(plans[j]->graph_stream, ev[0], 0));
                    TRY(solve_iter(plans[j], c[j], plans[j]->graph_stream));
                    DR_CUDA_TRY(cudaEventRecord(ev[j + 1], plans[j]->graph_stream));
                    DR_CUDA_TRY(cudaStreamWaitEvent(root, ev[j + 1], 0));
                }
                return DR_OK;
            },
            &exec);
        if (result != DR_OK) {
            // no graph: the same launches, one iteration at a time on each job's stream
            // (the root stream joins them afterwards)
            clear_error();
            result = DR_OK;
            for (int r = 0; r < reps && result == DR_OK; ++r)
                for (int j : act) {
                    result = solve_iter(plans[j], c[j], plans[j]->graph_stream);
                    if (result != DR_OK) break;
                }
            if (result != DR_OK) break;
            for (int j : act) c[j].done += reps;
            continue;
        }
        cudaError_t ce = cudaSuccess;
        for (int r = 0; r < reps && ce == cudaSuccess; ++r) ce = cudaGraphLaunch(exec, root);
        cudaGraphExecDestroy(exec);
        if (ce != cudaSuccess) {
            result = cuda_fail(ce, "admm_solve_batch: graph launch");
            break;
        }
        for (int j : act) c[j].done += reps;
    }
    // the jobs' own streams continue after the root stream's replays
    if (result == DR_OK && cudaEventRecord(ev[0], root) != cudaSuccess) result = fail(DR_ECUDA, "batch: join");
    for (int j = 0; j < n && result == DR_OK; ++j)
        if (cudaStreamWaitEvent(plans[j]->graph_stream, ev[0], 0) != cudaSuccess) result = fail(DR_ECUDA, "batch: join");
    for (int j = 0; j < n && result == DR_OK; ++j) result = solve_end(plans[j], c[j]);
    cudaStreamSynchronize(root);
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    cudaStreamDestroy(root);
    return result;
}

static dr_status check_params(const dr_solve_params &p) {
    if (p.algo != DR_ADMM_CG && p.algo != DR_CHAMBOLLE_POCK) return fail(DR_EINVAL, "admm_solve: bad algo");
    if (p.iters < 0 || (p.algo == DR_ADMM_CG && p.n_cg < 1)) return fail(DR_EINVAL, "admm_solve: bad iters/n_cg");
    if (!(p.lambda1 >= 0.0) || !(p.lambda2 >= 0.0) || !std::isfinite(p.lambda1) || !std::isfinite(p.lambda2) ||
        !std::isfinite(p.rho) || !std::isfinite(p.cp_theta) || !std::isfinite(p.op_norm))
        return fail(DR_EINVAL, "admm_solve: lambdas must be finite and >= 0");
    if (p.algo == DR_CHAMBOLLE_POCK && !(p.cp_theta >= 0.0 && p.cp_theta <= 1.0))
        return fail(DR_EINVAL, "admm_solve: cp_theta must be in [0, 1]");
    if (p.resume && !p.state) return fail(DR_EINVAL, "admm_solve: resume needs a state buffer");
    if (p.state && !is_device_ptr(p.state)) return fail(DR_EINVAL, "admm_solve: state must be device memory");
    return DR_OK;
}

}  // namespace dr

using namespace dr;

extern "C" {

size_t dr_plan_workspace_bytes(const dr_plan *P, dr_algo algo) { return P ? ws_bytes(P, algo, 1) : 0; }

size_t dr_plan_state_bytes(const dr_plan *P, dr_algo algo) {
    if (!P) return 0;
    const size_t cs = calc_size(P->prec), fs = field_size(P);
    if (algo == DR_ADMM_CG) return 2 * nf_elems(P) * fs;
    if (algo == DR_CHAMBOLLE_POCK) return nf_elems(P) * fs + (ng_elems(P) + nu_elems(P)) * cs;
    return 0;
}

dr_status admm_solve(dr_plan *P, const void *g, void *u, const dr_solve_params *prm) {
    clear_error();
    if (!P || !g || !u || !prm) return fail(DR_EINVAL, "admm_solve: NULL argument");
    TRY(check_params(*prm));
    TRY(ensure_ws(P, prm->algo, prm->iters));
    return solve(P, g, u, *prm);
}

dr_status admm_solve_batch(int njobs, dr_plan *const *plans, const void *const *g, void *const *u,
                           const dr_solve_params *params) {
    clear_error();
    if (njobs < 1 || !plans || !g || !u || !params) return fail(DR_EINVAL, "admm_solve_batch: bad arguments");
    for (int j = 0; j < njobs; ++j) {
        if (!plans[j] || !g[j] || !u[j]) return fail(DR_EINVAL, "admm_solve_batch: NULL job entry");
        if (plans[j]->device != plans[0]->device) return fail(DR_EINVAL, "admm_solve_batch: plans on different devices");
        for (int i = 0; i < j; ++i)
            if (plans[i] == plans[j]) return fail(DR_EINVAL, "admm_solve_batch: a plan appears twice");
        TRY(check_params(params[j]));
    }
    for (int j = 0; j < njobs; ++j) TRY(ensure_ws(plans[j], params[j].algo, params[j].iters));
    return solve_batch(njobs, plans, g, u, params);
}

}  // extern "C"
