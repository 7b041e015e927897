// projector.cu -- precision dispatch and C entry points of the dynamic
// projector pair (Sec. 4, Eqs. radapr and radadjapr).  The kernels live in
// projector_impl.cuh and are instantiated per precision in projector_*.cu.
#include <cmath>

#include "projector_impl.cuh"

namespace dr {

dr_status launch_fwd(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                     cudaStream_t st) {
    switch (P->prec) {
        case DR_F32: return ProjOps<float, float>::fwd(P, u, out, gm, mode, sigma, st);
        case DR_BF16_F32ACC: return ProjOps<bf16, float>::fwd(P, u, out, gm, mode, sigma, st);
        case DR_F64: return ProjOps<double, double>::fwd(P, u, out, gm, mode, sigma, st);
    }
    return fail(DR_EINVAL, "bad precision");
}

dr_status launch_adj(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                     cudaStream_t st) {
    switch (P->prec) {
        case DR_F32: return ProjOps<float, float>::adj(P, g, u, alpha, beta, u_calc, st);
        case DR_BF16_F32ACC: return ProjOps<bf16, float>::adj(P, g, u, alpha, beta, u_calc, st);
        case DR_F64: return ProjOps<double, double>::adj(P, g, u, alpha, beta, u_calc, st);
    }
    return fail(DR_EINVAL, "bad precision");
}

// Compute-typed variants for the solvers: all buffers are float (F32 and
// BF16 plans) or double (F64 plans).
dr_status launch_fwd_calc(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                          cudaStream_t st) {
    if (P->prec == DR_F64) return ProjOps<double, double>::fwd(P, u, out, gm, mode, sigma, st);
    return ProjOps<float, float>::fwd(P, u, out, gm, mode, sigma, st);
}

dr_status launch_adj_calc(dr_plan *P, const void *g, void *u, double alpha, double beta, cudaStream_t st) {
    if (P->prec == DR_F64) return ProjOps<double, double>::adj(P, g, u, alpha, beta, true, st);
    return ProjOps<float, float>::adj(P, g, u, alpha, beta, true, st);
}

}  // namespace dr

using namespace dr;

extern "C" {

dr_status dyn_radon_fwd(dr_plan *P, const void *u, void *g) {
    clear_error();
    if (!P || !u || !g) return fail(DR_EINVAL, "dyn_radon_fwd: NULL argument");
    return launch_fwd(P, u, g, nullptr, 0, 0.0, P->stream);
}

dr_status dyn_radon_adj(dr_plan *P, const void *g, void *u, double beta) {
    clear_error();
    if (!P || !u || !g) return fail(DR_EINVAL, "dyn_radon_adj: NULL argument");
    if (!std::isfinite(beta)) return fail(DR_EINVAL, "dyn_radon_adj: beta must be finite");
    return launch_adj(P, g, u, 1.0, beta, false, P->stream);
}

}  // extern "C"
