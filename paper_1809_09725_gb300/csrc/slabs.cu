// slabs.cu -- Chambolle-Pock (Sec. 3, Fig. 2) on a volume that stays in host
// memory and is streamed through the GPU in slabs of slices (Sec. 6).
//
// The paper splits the volume into sets of slices, moves each set to the GPU
// with the slice before and after it for the z derivatives, and overlaps the
// host-to-device copies, the computation and the device-to-host copies on
// three streams.  Here every iteration walks the slabs z0 = 0, S, 2S, ... in
// order; slab [z0, z1) needs
//   * u~ on [z0, z1] (the slice above feeds the forward z difference of D;
//     when the volume has at most S+1 slabs, after the first iteration it
//     comes from a device copy that the slab above left behind, so a slab's
//     copy-in waits only for its own copy-out; with more slabs the halo
//     copies would outgrow a slab and the halo is re-read from the host),
//   * the NEW dual h2 on slice z0-1 (the backward difference of D^T): the
//     previous slab computed it, and it is carried over on the device instead
//     of being re-read from the host (where the old value is already gone),
//   * for the objective, the NEW u on slice z0-1 (carried the same way).
// Every kernel computes each output element from the same inputs in the same
// order as the whole-volume solver, so with the same operator norm the
// result is the in-core Chambolle-Pock result bit for bit.
//
// Three device stages rotate: while slab q computes, slab q+1 is copied in
// and slab q-1 is copied out, and the copy-in of q+1 need not wait for the
// copy-out of q-1.  A slab's copy-in waits for the copy-out of the slab that
// last used its stage and, from the previous iteration, of the slab above it
// (which wrote the halo slice it reads).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "dr_device.cuh"

namespace dr {

dr_status launch_fwd_calc(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                          cudaStream_t st);
dr_status launch_adj_calc(dr_plan *P, const void *g, void *u, double alpha, double beta, cudaStream_t st);
dr_status launch_dot_obj(dr_plan *P, const void *a, const void *b, size_t n, double *obj, int row_off, int col,
                         cudaStream_t st);
dr_status launch_set_iter(dr_plan *P, int value, cudaStream_t st);
dr_status launch_pow_init(dr_plan *P, void *x, size_t n, size_t first, cudaStream_t st);
dr_status launch_convert_bf16(dr_plan *P, const void *in, void *out, size_t n, bool to_bf16, cudaStream_t st);

#define STRY(...)                      \
    do {                               \
        dr_status _s = (__VA_ARGS__);  \
        if (_s != DR_OK) return _s;    \
    } while (0)

namespace {

constexpr int kStages = 3;

// Sizes of one slab problem (elements per slice of each array).
struct SlabDims {
    size_t A;    // nx * ny
    size_t um;   // A * m            coefficients per slice
    size_t gk;   // K * ns           data per slice
    size_t f4;   // A * nt * 4       dual field per slice
    size_t cs, es;
    int S, nz, nslab;
};

SlabDims dims_of(const dr_plan *P, int S, int nz_total) {
    SlabDims d;
    d.A = (size_t)P->nx * P->ny;
    d.um = d.A * P->m;
    d.gk = (size_t)P->K * P->ns;
    d.f4 = d.A * P->nt * 4;
    d.cs = calc_size(P->prec);
    d.es = elem_size(P->prec);
    d.S = S;
    d.nz = nz_total;
    d.nslab = (nz_total + S - 1) / S;
    return d;
}

size_t fold_scratch_bytes(const dr_plan *P, int S) {
    if (P->fold_U == 0) return 0;
    const int M = P->M;
    const int MS = M <= 4 ? 4 : ((M % 8 == 0) ? M + 4 : M);
    return sizeof(float) * (size_t)S * P->fold_U * P->ns * MS;
}

// Device buffers of the streamed solve.
struct Stage {
    void *U = nullptr;   // [1 + S] slices: u carry (slice z0-1) + body
    void *UT = nullptr;  // [S + 1]: body + halo above
    void *H1 = nullptr;  // [S] data slices
    void *G = nullptr;   // [S] data slices, compute typed
    void *GR = nullptr;  // [S] data slices, bf16 (BF16 plans)
    void *H2 = nullptr;  // [1 + S]: carry (slice z0-1) + body
};

struct Buffers {
    Stage st[kStages];
    void *Abuf = nullptr, *GD = nullptr;          // R* h1 [S], R u - g [S]
    void *carry_h2 = nullptr, *carry_u = nullptr;  // one slice each
    void *halo_ut = nullptr;                       // [nslab-1] u~ on the first slice of slabs 1..
    void *gt = nullptr;                            // folded-data scratch for S slices
    double *obj = nullptr;
    std::vector<void *> all;
    size_t bytes = 0;
    bool ok = true;
    void *get(size_t n) {
        void *p = nullptr;
        if (!ok) return nullptr;
        if (cudaMalloc(&p, std::max<size_t>(n, 16)) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
            return nullptr;
        }
        all.push_back(p);
        bytes += n;
        return p;
    }
    ~Buffers() {
        for (void *p : all) cudaFree(p);
    }
};

// Device copies of the u~ halo slices: worth it (and cheap) with few slabs.
bool device_halo(const SlabDims &d) { return d.nslab > 1 && d.nslab - 1 <= d.S; }

size_t device_bytes(const dr_plan *P, const SlabDims &d, bool bf, bool power, int rows) {
    const size_t S = d.S, cs = d.cs;
    size_t b = 0;
    b += kStages * ((S + 1) * d.um * cs * 2 + S * d.gk * cs * 2 + (S + 1) * d.f4 * cs);
    if (bf) b += kStages * S * d.gk * 2;
    b += S * d.um * cs + S * d.gk * cs + d.f4 * cs + d.um * cs;
    if (device_halo(d)) b += (size_t)(d.nslab - 1) * d.um * cs;
    if (!P->d_gt) b += fold_scratch_bytes(P, d.S);
    if (power) b += kStages * ((S + 2) * d.um * cs + S * d.um * cs);
    b += sizeof(double) * 3 * (size_t)(rows + 1);
    return b;
}

// Three streams, per-stage and per-slab events.
struct Pipe {
    cudaStream_t hs = nullptr, cs = nullptr, ds = nullptr;
    cudaEvent_t ev_h2d[kStages] = {}, ev_comp[kStages] = {}, ev_d2h[kStages] = {};
    std::vector<cudaEvent_t> ev_slab;
    long long q = 0;     // slabs issued so far (selects the stage)
    bool first = true;   // no previous pass to wait for
    dr_status init(int device, int nslab) {
        (void)device;
        DR_CUDA_TRY(cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking));
        DR_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        DR_CUDA_TRY(cudaStreamCreateWithFlags(&ds, cudaStreamNonBlocking));
        for (int i = 0; i < kStages; ++i) {
            DR_CUDA_TRY(cudaEventCreateWithFlags(&ev_h2d[i], cudaEventDisableTiming));
            DR_CUDA_TRY(cudaEventCreateWithFlags(&ev_comp[i], cudaEventDisableTiming));
            DR_CUDA_TRY(cudaEventCreateWithFlags(&ev_d2h[i], cudaEventDisableTiming));
        }
        ev_slab.assign(nslab, nullptr);
        for (auto &e : ev_slab) DR_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        return DR_OK;
    }
    ~Pipe() {
        for (cudaStream_t s : {hs, cs, ds})
            if (s) cudaStreamSynchronize(s);
        for (int i = 0; i < kStages; ++i)
            for (cudaEvent_t e : {ev_h2d[i], ev_comp[i], ev_d2h[i]})
                if (e) cudaEventDestroy(e);
        for (auto e : ev_slab)
            if (e) cudaEventDestroy(e);
        for (cudaStream_t s : {hs, cs, ds})
            if (s) cudaStreamDestroy(s);
    }
    dr_status sync() {
        DR_CUDA_TRY(cudaStreamSynchronize(hs));
        DR_CUDA_TRY(cudaStreamSynchronize(cs));
        DR_CUDA_TRY(cudaStreamSynchronize(ds));
        return DR_OK;
    }
    // One pass over all slabs: copy in, compute, copy out, overlapped.
    // halo_from_host: a slab's copy-in also reads the slice above it from the
    // host, so it waits for the previous pass's copy-out of the next slab too.
    dr_status pass(int nslab, bool halo_from_host, const std::function<dr_status(int, int, cudaStream_t)> &h2d,
                   const std::function<dr_status(int, int, cudaStream_t)> &comp,
                   const std::function<dr_status(int, int, cudaStream_t)> &d2h) {
        for (int s = 0; s < nslab; ++s, ++q) {
            const int b = (int)(q % kStages);
            if (q >= kStages) DR_CUDA_TRY(cudaStreamWaitEvent(hs, ev_d2h[b], 0));
            if (!first)
                DR_CUDA_TRY(cudaStreamWaitEvent(hs, ev_slab[halo_from_host ? std::min(s + 1, nslab - 1) : s], 0));
            STRY(h2d(s, b, hs));
            DR_CUDA_TRY(cudaEventRecord(ev_h2d[b], hs));
            DR_CUDA_TRY(cudaStreamWaitEvent(cs, ev_h2d[b], 0));
            STRY(comp(s, b, cs));
            DR_CUDA_TRY(cudaEventRecord(ev_comp[b], cs));
            DR_CUDA_TRY(cudaStreamWaitEvent(ds, ev_comp[b], 0));
            STRY(d2h(s, b, ds));
            DR_CUDA_TRY(cudaEventRecord(ev_d2h[b], ds));
            DR_CUDA_TRY(cudaEventRecord(ev_slab[s], ds));
        }
        first = false;
        return DR_OK;
    }
};

// Pinned host buffer.
struct HostBuf {
    void *p = nullptr;
    size_t n = 0;
    dr_status alloc(size_t bytes) {
        n = bytes;
        DR_CUDA_TRY(cudaHostAlloc(&p, std::max<size_t>(bytes, 16), cudaHostAllocPortable));
        return DR_OK;
    }
    ~HostBuf() {
        if (p) cudaFreeHost(p);
    }
    unsigned char *at(size_t off) const { return (unsigned char *)p + off; }
};

// Restores the plan fields a slab solve changes.
struct PlanScope {
    dr_plan *P;
    int nz;
    void *gt;
    bool fields_bf16;
    // the slab solver keeps float dual fields (its halo copies move floats)
    explicit PlanScope(dr_plan *p) : P(p), nz(p->nz), gt(p->d_gt), fields_bf16(p->fields_bf16) {
        P->split_off = true;
        P->fields_bf16 = false;
    }
    ~PlanScope() {
        P->split_off = false;
        P->fields_bf16 = fields_bf16;
        P->nz = nz;
        P->z_open_lo = P->z_open_hi = 0;
        P->d_gt = gt;
    }
};

bool is_pinned_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

bool is_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// bf16 <-> float on the host (round to nearest even, NaN kept quiet).
inline float bf16_to_float(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
inline uint16_t float_to_bf16(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

}  // namespace

static dr_status slab_solve(dr_plan *P, const void *g_user, void *u_user, const dr_solve_params &prm, int S,
                            size_t *bytes_only) {
    const int nz = P->nz;
    S = std::min(S, nz);
    const SlabDims d = dims_of(P, S, nz);
    const bool bf = P->prec == DR_BF16_F32ACC;
    const bool want_obj = prm.objective_out != nullptr;
    const bool power = !(prm.op_norm > 0.0);
    const int rows = std::max(prm.iters * d.nslab, power ? std::max(prm.power_iters, 1) * d.nslab + d.nslab : 0);
    if (bytes_only) {
        *bytes_only = device_bytes(P, d, bf, power, rows);
        return DR_OK;
    }
    if (is_device(g_user) || is_device(u_user))
        return fail(DR_EINVAL, "cp_solve_slabs: g and u must be host buffers (admm_solve takes device buffers)");

    PlanScope scope(P);
    Buffers B;
    const size_t cs = d.cs;
    for (int i = 0; i < kStages; ++i) {
        Stage &t = B.st[i];
        t.U = B.get((S + 1) * d.um * cs);
        t.UT = B.get((S + 1) * d.um * cs);
        t.H1 = B.get(S * d.gk * cs);
        t.G = B.get(S * d.gk * cs);
        if (bf) t.GR = B.get(S * d.gk * 2);
        t.H2 = B.get((S + 1) * d.f4 * cs);
    }
    B.Abuf = B.get(S * d.um * cs);
    B.GD = B.get(S * d.gk * cs);
    B.carry_h2 = B.get(d.f4 * cs);
    B.carry_u = B.get(d.um * cs);
    const bool dev_halo = device_halo(d);
    if (dev_halo) B.halo_ut = B.get((size_t)(d.nslab - 1) * d.um * cs);
    if (!P->d_gt && P->fold_U > 0) B.gt = B.get(fold_scratch_bytes(P, S));
    B.obj = (double *)B.get(sizeof(double) * 3 * (size_t)(rows + 1));
    if (!B.ok) return fail(DR_ENOMEM, "cp_solve_slabs: device allocation failed (use a thinner slab)");
    if (B.gt) P->d_gt = B.gt;

    // the variants: timed on one slab's geometry unless chosen explicitly
    P->nz = S;
    if (!P->tuned && (P->var_fwd < 0 || P->var_adj < 0)) STRY(autotune(P, B.Abuf, B.GD));

    // ---- host state ----
    const size_t nu = (size_t)nz * d.um, ng = (size_t)nz * d.gk, nf = (size_t)nz * d.f4;
    HostBuf uh, uth, h1h, h2h, gh, yh;
    STRY(uh.alloc(nu * cs));
    STRY(uth.alloc(nu * cs));
    STRY(h1h.alloc(ng * cs));
    STRY(h2h.alloc(nf * cs));
    const unsigned char *g_host = (const unsigned char *)g_user;
    if (!is_pinned_host(g_user)) {
        STRY(gh.alloc(ng * d.es));
        std::memcpy(gh.p, g_user, ng * d.es);
        g_host = gh.at(0);
    }
    if (bf) {
        const uint16_t *src = (const uint16_t *)u_user;
        float *dst = (float *)uh.p;
        for (size_t i = 0; i < nu; ++i) dst[i] = bf16_to_float(src[i]);
    } else {
        std::memcpy(uh.p, u_user, nu * cs);
    }

    Pipe pipe;
    STRY(pipe.init(P->device, d.nslab));
    auto z0_of = [&](int s) { return s * S; };
    auto n_of = [&](int s) { return std::min(S, nz - s * S); };

    // ---- operator norm ||[R; D]|| by power iteration, streamed ----
    double L = prm.op_norm;
    if (power) {
        const int iters = prm.power_iters > 0 ? prm.power_iters : 100;
        void *X[kStages], *Y[kStages];
        for (int i = 0; i < kStages; ++i) {
            X[i] = B.get((S + 2) * d.um * cs);
            Y[i] = B.get(S * d.um * cs);
        }
        if (!B.ok) return fail(DR_ENOMEM, "cp_solve_slabs: device allocation failed (use a thinner slab)");
        STRY(yh.alloc(nu * cs));
        HostBuf *yin = &uth, *yout = &yh;  // uth is free until the iterations start
        std::vector<double> hrow(3 * (size_t)(d.nslab + 1));
        // ||x0||^2 of the SplitMix start, slab by slab
        DR_CUDA_TRY(cudaMemsetAsync(B.obj, 0, sizeof(double) * 3 * (size_t)(d.nslab + 1), pipe.cs));
        for (int s = 0; s < d.nslab; ++s) {
            const size_t n = (size_t)n_of(s) * d.um;
            STRY(launch_pow_init(P, X[0], n, (size_t)z0_of(s) * d.um, pipe.cs));
            STRY(launch_set_iter(P, s, pipe.cs));
            STRY(launch_dot_obj(P, X[0], X[0], n, B.obj, 1, 0, pipe.cs));
        }
        DR_CUDA_TRY(cudaMemcpyAsync(hrow.data(), B.obj, sizeof(double) * hrow.size(), cudaMemcpyDeviceToHost, pipe.cs));
        STRY(pipe.sync());
        double lam = 0.0;
        for (int s = 0; s < d.nslab; ++s) lam += hrow[3 * (size_t)(s + 1)];
        for (int it = 0; it < iters; ++it) {
            const double alpha = lam > 0.0 ? 1.0 / std::sqrt(lam) : 0.0;
            DR_CUDA_TRY(cudaMemsetAsync(B.obj, 0, sizeof(double) * 3 * (size_t)(d.nslab + 1), pipe.cs));
            auto lo_h = [&](int s) { return s > 0 ? 1 : 0; };
            auto hi_h = [&](int s) { return z0_of(s) + n_of(s) < nz ? 1 : 0; };
            STRY(pipe.pass(
                d.nslab, true,
                [&](int s, int b, cudaStream_t st) -> dr_status {
                    if (it == 0) return DR_OK;  // the start vector is generated on the device
                    const size_t first = (size_t)(z0_of(s) - lo_h(s)) * d.um;
                    const size_t cnt = (size_t)(n_of(s) + lo_h(s) + hi_h(s)) * d.um;
                    DR_CUDA_TRY(cudaMemcpyAsync(X[b], yin->at(first * cs), cnt * cs, cudaMemcpyHostToDevice, st));
                    return DR_OK;
                },
                [&](int s, int b, cudaStream_t st) -> dr_status {
                    const int ns_ = n_of(s), lo = lo_h(s), hi = hi_h(s);
                    if (it == 0)
                        STRY(launch_pow_init(P, X[b], (size_t)(ns_ + lo + hi) * d.um, (size_t)(z0_of(s) - lo) * d.um,
                                             st));
                    void *xb = (unsigned char *)X[b] + (size_t)lo * d.um * cs;
                    P->nz = ns_;
                    STRY(launch_fwd_calc(P, xb, B.GD, nullptr, 0, 0.0, st));
                    STRY(launch_adj_calc(P, B.GD, Y[b], alpha, 0.0, st));
                    P->z_open_lo = lo;
                    P->z_open_hi = hi;
                    dr_status r = launch_lap(P, xb, Y[b], alpha, 1.0, prm.lambda2, 0, st);
                    P->z_open_lo = P->z_open_hi = 0;
                    STRY(r);
                    STRY(launch_set_iter(P, s, st));
                    return launch_dot_obj(P, Y[b], Y[b], (size_t)ns_ * d.um, B.obj, 1, 0, st);
                },
                [&](int s, int b, cudaStream_t st) -> dr_status {
                    DR_CUDA_TRY(cudaMemcpyAsync(yout->at((size_t)z0_of(s) * d.um * cs), Y[b],
                                                (size_t)n_of(s) * d.um * cs, cudaMemcpyDeviceToHost, st));
                    return DR_OK;
                }));
            DR_CUDA_TRY(cudaMemcpyAsync(hrow.data(), B.obj, sizeof(double) * hrow.size(), cudaMemcpyDeviceToHost,
                                        pipe.cs));
            STRY(pipe.sync());
            lam = 0.0;
            for (int s = 0; s < d.nslab; ++s) lam += hrow[3 * (size_t)(s + 1)];
            std::swap(yin, yout);
            pipe.first = true;  // the next pass reads the other host buffer
        }
        L = std::sqrt(std::sqrt(lam));
    }
    if (!(L > 0.0) || !std::isfinite(L)) return fail(DR_EINVAL, "cp_solve_slabs: operator norm is zero");
    if (prm.op_norm_out) *prm.op_norm_out = L;
    const double sigma = 0.99 / L, tau = 0.99 / L;

    // ---- Chambolle-Pock iterations ----
    std::memcpy(uth.p, uh.p, nu * cs);
    std::memset(h1h.p, 0, ng * cs);
    std::memset(h2h.p, 0, nf * cs);
    DR_CUDA_TRY(cudaMemsetAsync(B.obj, 0, sizeof(double) * 3 * (size_t)(rows + 1), pipe.cs));
    pipe.first = true;
    for (int it = 0; it < prm.iters; ++it) {
        STRY(pipe.pass(
            d.nslab, it == 0 || !dev_halo,
            [&](int s, int b, cudaStream_t st) -> dr_status {
                const Stage &t = B.st[b];
                const size_t z0 = z0_of(s), n = n_of(s);
                const size_t hi = ((it == 0 || !dev_halo) && z0 + n < (size_t)nz) ? 1 : 0;
                DR_CUDA_TRY(cudaMemcpyAsync((unsigned char *)t.U + d.um * cs, uh.at(z0 * d.um * cs), n * d.um * cs,
                                            cudaMemcpyHostToDevice, st));
                DR_CUDA_TRY(cudaMemcpyAsync(t.UT, uth.at(z0 * d.um * cs), (n + hi) * d.um * cs, cudaMemcpyHostToDevice,
                                            st));
                DR_CUDA_TRY(cudaMemcpyAsync(t.H1, h1h.at(z0 * d.gk * cs), n * d.gk * cs, cudaMemcpyHostToDevice, st));
                DR_CUDA_TRY(cudaMemcpyAsync((unsigned char *)t.H2 + d.f4 * cs, h2h.at(z0 * d.f4 * cs), n * d.f4 * cs,
                                            cudaMemcpyHostToDevice, st));
                DR_CUDA_TRY(cudaMemcpyAsync(bf ? t.GR : t.G, g_host + z0 * d.gk * d.es, n * d.gk * d.es,
                                            cudaMemcpyHostToDevice, st));
                return DR_OK;
            },
            [&](int s, int b, cudaStream_t st) -> dr_status {
                const Stage &t = B.st[b];
                const int n = n_of(s);
                const bool last = s == d.nslab - 1;
                const int hi = last ? 0 : 1;
                void *Ub = (unsigned char *)t.U + d.um * cs;
                void *H2b = (unsigned char *)t.H2 + d.f4 * cs;
                if (bf) STRY(launch_convert_bf16(P, t.GR, t.G, (size_t)n * d.gk, false, st));
                if (s > 0) {
                    DR_CUDA_TRY(cudaMemcpyAsync(t.H2, B.carry_h2, d.f4 * cs, cudaMemcpyDeviceToDevice, st));
                    if (want_obj) DR_CUDA_TRY(cudaMemcpyAsync(t.U, B.carry_u, d.um * cs, cudaMemcpyDeviceToDevice, st));
                }
                // the halo u~ (slice z1, as of the previous iteration) from the device copy
                if (dev_halo && it > 0 && !last)
                    DR_CUDA_TRY(cudaMemcpyAsync((unsigned char *)t.UT + (size_t)n * d.um * cs,
                                                (unsigned char *)B.halo_ut + (size_t)s * d.um * cs, d.um * cs,
                                                cudaMemcpyDeviceToDevice, st));
                P->nz = n;
                // Fig. 2 steps 3-6 on the slab
                STRY(launch_fwd_calc(P, t.UT, t.H1, t.G, 2, sigma, st));
                P->z_open_hi = hi;
                dr_status r = launch_cp_dual(P, t.UT, H2b, sigma, prm.lambda1, prm.lambda2, st);
                P->z_open_hi = 0;
                STRY(r);
                STRY(launch_adj_calc(P, t.H1, B.Abuf, 1.0, 0.0, st));
                P->z_open_lo = s > 0 ? 1 : 0;
                P->z_open_hi = hi;
                r = launch_cp_primal(P, Ub, t.UT, B.Abuf, H2b, tau, prm.cp_theta, prm.lambda2, st);
                P->z_open_lo = P->z_open_hi = 0;
                STRY(r);
                if (!last) {
                    DR_CUDA_TRY(cudaMemcpyAsync(B.carry_h2, (unsigned char *)H2b + (size_t)(n - 1) * d.f4 * cs,
                                                d.f4 * cs, cudaMemcpyDeviceToDevice, st));
                }
                // the new u~ on this slab's first slice is the next iteration's halo of the slab below
                if (dev_halo && s > 0)
                    DR_CUDA_TRY(cudaMemcpyAsync((unsigned char *)B.halo_ut + (size_t)(s - 1) * d.um * cs, t.UT,
                                                d.um * cs, cudaMemcpyDeviceToDevice, st));
                if (want_obj) {
                    if (!last)
                        DR_CUDA_TRY(cudaMemcpyAsync(B.carry_u, (unsigned char *)Ub + (size_t)(n - 1) * d.um * cs,
                                                    d.um * cs, cudaMemcpyDeviceToDevice, st));
                    const int row = it * d.nslab + s;  // written at row + 1
                    STRY(launch_set_iter(P, row, st));
                    STRY(launch_fwd_calc(P, Ub, B.GD, t.G, 1, 0.0, st));
                    STRY(launch_dot_obj(P, B.GD, B.GD, (size_t)n * d.gk, B.obj, 1, 0, st));
                    // TV of slices [z0 - 1, z1 - 1) (of [0, z1 - 1) for the first slab, up to
                    // nz for the last): every forward z difference sees the new u on both sides
                    const int lo = s > 0 ? 0 : 1;
                    const int hi_idx = last ? n + 1 : n;
                    if (hi_idx > lo) {
                        P->nz = hi_idx - lo;
                        P->z_open_hi = hi;
                        r = launch_tv_sum(P, (unsigned char *)t.U + (size_t)lo * d.um * cs, prm.lambda2, B.obj + 3, st);
                        P->z_open_hi = 0;
                        STRY(r);
                    }
                }
                return DR_OK;
            },
            [&](int s, int b, cudaStream_t st) -> dr_status {
                const Stage &t = B.st[b];
                const size_t z0 = z0_of(s), n = n_of(s);
                DR_CUDA_TRY(cudaMemcpyAsync(uh.at(z0 * d.um * cs), (unsigned char *)t.U + d.um * cs, n * d.um * cs,
                                            cudaMemcpyDeviceToHost, st));
                DR_CUDA_TRY(cudaMemcpyAsync(uth.at(z0 * d.um * cs), t.UT, n * d.um * cs, cudaMemcpyDeviceToHost, st));
                DR_CUDA_TRY(cudaMemcpyAsync(h1h.at(z0 * d.gk * cs), t.H1, n * d.gk * cs, cudaMemcpyDeviceToHost, st));
                DR_CUDA_TRY(cudaMemcpyAsync(h2h.at(z0 * d.f4 * cs), (unsigned char *)t.H2 + d.f4 * cs, n * d.f4 * cs,
                                            cudaMemcpyDeviceToHost, st));
                return DR_OK;
            }));
    }
    std::vector<double> hobj;
    if (want_obj && prm.iters > 0) {
        hobj.resize(3 * (size_t)(rows + 1));
        DR_CUDA_TRY(cudaMemcpyAsync(hobj.data(), B.obj, sizeof(double) * hobj.size(), cudaMemcpyDeviceToHost,
                                    pipe.cs));
    }
    STRY(pipe.sync());
    int flag = 0;
    DR_CUDA_TRY(cudaMemcpy(&flag, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(P->d_status, 0, sizeof(int));
        return fail(DR_ETIMEOUT, "cp_solve_slabs: a bounded device-side wait gave up");
    }
    bool finite = true;
    if (bf) {
        const float *src = (const float *)uh.p;
        uint16_t *dst = (uint16_t *)u_user;
        for (size_t i = 0; i < nu; ++i) {
            if (!std::isfinite(src[i])) finite = false;
            dst[i] = float_to_bf16(src[i]);
        }
    } else {
        std::memcpy(u_user, uh.p, nu * cs);
        if (cs == 4) {
            for (size_t i = 0; i < nu && finite; ++i) finite = std::isfinite(((const float *)uh.p)[i]);
        } else {
            for (size_t i = 0; i < nu && finite; ++i) finite = std::isfinite(((const double *)uh.p)[i]);
        }
    }
    for (int it = 0; it < prm.iters && !hobj.empty(); ++it) {
        double fid = 0.0, tv = 0.0;
        for (int s = 0; s < d.nslab; ++s) {
            const double *row = &hobj[3 * (size_t)(it * d.nslab + s + 1)];
            fid += row[0];
            tv += row[1];
        }
        prm.objective_out[it] = 0.5 * fid + prm.lambda1 * tv;
        if (!std::isfinite(prm.objective_out[it])) finite = false;
    }
    if (!finite) return fail(DR_ENOTCONV, "cp_solve_slabs: non-finite values (check the data for NaN/Inf)");
    return DR_OK;
}

}  // namespace dr

using namespace dr;

extern "C" {

dr_status cp_solve_slabs(dr_plan *P, const void *g, void *u, const dr_solve_params *prm, int slab_nz) {
    clear_error();
    if (!P || !g || !u || !prm) return fail(DR_EINVAL, "cp_solve_slabs: NULL argument");
    if (prm->algo != DR_CHAMBOLLE_POCK)
        return fail(DR_EINVAL,
                    "cp_solve_slabs: slab streaming runs Chambolle-Pock (ADMM-CG needs whole-volume inner products "
                    "inside every CG step)");
    if (slab_nz < 1) return fail(DR_EINVAL, "cp_solve_slabs: slab_nz must be >= 1");
    if (prm->state || prm->resume) return fail(DR_EINVAL, "cp_solve_slabs: takes no solver state buffer");
    if (prm->iters < 0) return fail(DR_EINVAL, "cp_solve_slabs: iters must be >= 0");
    if (!(prm->lambda1 >= 0.0) || !(prm->lambda2 >= 0.0) || !std::isfinite(prm->lambda1) ||
        !std::isfinite(prm->lambda2) || !std::isfinite(prm->op_norm))
        return fail(DR_EINVAL, "cp_solve_slabs: lambdas must be finite and >= 0");
    if (!(prm->cp_theta >= 0.0 && prm->cp_theta <= 1.0))
        return fail(DR_EINVAL, "cp_solve_slabs: cp_theta must be in [0, 1]");
    DR_CUDA_TRY(cudaStreamSynchronize(P->stream));
    return slab_solve(P, g, u, *prm, slab_nz, nullptr);
}

size_t cp_solve_slabs_device_bytes(dr_plan *P, int slab_nz, const dr_solve_params *prm) {
    if (!P || !prm || slab_nz < 1) return 0;
    size_t b = 0;
    if (slab_solve(P, nullptr, nullptr, *prm, slab_nz, &b) != DR_OK) return 0;
    return b;
}

}  // extern "C"
