// tv.cu -- precision dispatch and C entry points of the 4D TV kernels
// (D = nabla_{lambda2} o PhiF of Eq. TV1, its adjoint, the ADMM prox).
#include <cmath>

#include "tv_impl.cuh"

namespace dr {

dr_status launch_grad(dr_plan *P, const void *u, bool calc, void *p, double lambda2, cudaStream_t st) {
    if (P->prec == DR_F64) return TvOps<double, double>::grad(P, u, p, lambda2, st);
    if (P->prec == DR_BF16_F32ACC && !calc) return TvOps<float, bf16>::grad(P, u, p, lambda2, st);
    return TvOps<float, float>::grad(P, u, p, lambda2, st);
}

dr_status launch_grad_adj(dr_plan *P, const void *p, void *u, bool calc, double lambda2, double alpha,
                          double beta, cudaStream_t st) {
    if (calc && P->fields_bf16) return TvFieldsBF16::grad_adj(P, p, u, lambda2, alpha, beta, st);
    if (P->prec == DR_F64) return TvOps<double, double>::grad_adj(P, p, u, calc, lambda2, alpha, beta, st);
    if (P->prec == DR_BF16_F32ACC && !calc)
        return TvOps<float, bf16>::grad_adj(P, p, u, false, lambda2, alpha, beta, st);
    return TvOps<float, float>::grad_adj(P, p, u, calc, lambda2, alpha, beta, st);
}

dr_status launch_prox(dr_plan *P, const void *u, bool calc, void *mu, void *w, double rho, double lambda1,
                      double lambda2, double *obj_row, cudaStream_t st) {
    if (calc && P->fields_bf16) return TvFieldsBF16::prox(P, u, mu, w, rho, lambda1, lambda2, obj_row, st);
    if (P->prec == DR_F64) return TvOps<double, double>::prox(P, u, mu, w, rho, lambda1, lambda2, obj_row, st);
    if (P->prec == DR_BF16_F32ACC && !calc)
        return TvOps<float, bf16>::prox(P, u, mu, w, rho, lambda1, lambda2, obj_row, st);
    return TvOps<float, float>::prox(P, u, mu, w, rho, lambda1, lambda2, obj_row, st);
}

dr_status launch_lap(dr_plan *P, const void *x, void *out, double alpha, double beta, double lambda2, int cg_step,
                     cudaStream_t st) {
    if (P->prec == DR_F64) return TvCalc<double>::lap(P, x, out, nullptr, alpha, beta, lambda2, cg_step, st);
    return TvCalc<float>::lap(P, x, out, nullptr, alpha, beta, lambda2, cg_step, st);
}

// r = r + rho (D^T w - D^T D u); p = r; rr = <r, r>; active = 1.
dr_status launch_rhs(dr_plan *P, const void *u, const void *w, void *r, void *p, double rho, double lambda2,
                     cudaStream_t st) {
    dr_status s = launch_grad_adj(P, w, r, true, lambda2, rho, 1.0, st);
    if (s != DR_OK) return s;
    if (P->prec == DR_F64) return TvCalc<double>::lap(P, u, r, p, -rho, 1.0, lambda2, 2, st);
    return TvCalc<float>::lap(P, u, r, p, -rho, 1.0, lambda2, 2, st);
}

dr_status launch_cp_dual(dr_plan *P, const void *ut, void *h2, double sigma, double lambda1, double lambda2,
                         cudaStream_t st) {
    if (P->fields_bf16) return TvFieldsBF16::cp_dual(P, ut, h2, sigma, lambda1, lambda2, st);
    if (P->prec == DR_F64) return TvCalc<double>::cp_dual(P, ut, h2, sigma, lambda1, lambda2, st);
    return TvCalc<float>::cp_dual(P, ut, h2, sigma, lambda1, lambda2, st);
}

dr_status launch_cp_primal(dr_plan *P, void *u, void *ut, const void *a, const void *h2, double tau, double theta,
                           double lambda2, cudaStream_t st) {
    if (P->fields_bf16) return TvFieldsBF16::cp_primal(P, u, ut, a, h2, tau, theta, lambda2, st);
    if (P->prec == DR_F64) return TvCalc<double>::cp_primal(P, u, ut, a, h2, tau, theta, lambda2, st);
    return TvCalc<float>::cp_primal(P, u, ut, a, h2, tau, theta, lambda2, st);
}

dr_status launch_tv_sum(dr_plan *P, const void *u, double lambda2, double *obj, cudaStream_t st) {
    if (P->prec == DR_F64) return TvCalc<double>::tv_sum(P, u, lambda2, obj, st);
    return TvCalc<float>::tv_sum(P, u, lambda2, obj, st);
}

}  // namespace dr

using namespace dr;

extern "C" {

dr_status tv4d_grad(dr_plan *P, const void *u, void *p, double lambda2) {
    clear_error();
    if (!P || !u || !p) return fail(DR_EINVAL, "tv4d_grad: NULL argument");
    if (!(lambda2 >= 0.0) || !std::isfinite(lambda2)) return fail(DR_EINVAL, "tv4d_grad: lambda2 must be >= 0");
    return launch_grad(P, u, false, p, lambda2, P->stream);
}

dr_status tv4d_grad_adj(dr_plan *P, const void *p, void *u, double lambda2, double beta) {
    clear_error();
    if (!P || !u || !p) return fail(DR_EINVAL, "tv4d_grad_adj: NULL argument");
    if (!(lambda2 >= 0.0) || !std::isfinite(lambda2) || !std::isfinite(beta))
        return fail(DR_EINVAL, "tv4d_grad_adj: bad lambda2/beta");
    return launch_grad_adj(P, p, u, false, lambda2, 1.0, beta, P->stream);
}

dr_status tv4d_normal(dr_plan *P, const void *x, void *out, double lambda2, double beta) {
    clear_error();
    if (!P || !x || !out) return fail(DR_EINVAL, "tv4d_normal: NULL argument");
    if (x == out) return fail(DR_EINVAL, "tv4d_normal: x and out must be distinct buffers");
    if (!(lambda2 >= 0.0) || !std::isfinite(lambda2) || !std::isfinite(beta))
        return fail(DR_EINVAL, "tv4d_normal: bad lambda2/beta");
    return launch_lap(P, x, out, 1.0, beta, lambda2, 0, P->stream);
}

dr_status tv4d_prox(dr_plan *P, const void *u, void *mu, void *w, double rho, double lambda1, double lambda2,
                    double *primal_res) {
    clear_error();
    if (!P || !u || !mu || !w) return fail(DR_EINVAL, "tv4d_prox: NULL argument");
    if (!(rho > 0.0) || !std::isfinite(rho) || !(lambda1 >= 0.0) || !std::isfinite(lambda1) || !(lambda2 >= 0.0) ||
        !std::isfinite(lambda2))
        return fail(DR_EINVAL, "tv4d_prox: need rho > 0, lambda1 >= 0, lambda2 >= 0 (finite)");
    dr_status s = launch_prox(P, u, false, mu, w, rho, lambda1, lambda2, nullptr, P->stream);
    if (s != DR_OK || !primal_res) return s;
    DevScalars hs;
    cudaError_t e = cudaMemcpyAsync(&hs, P->d_scal, sizeof(hs), cudaMemcpyDeviceToHost, P->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_fail(e, "tv4d_prox: read residual");
    *primal_res = std::sqrt(hs.acc2);
    return DR_OK;
}

}  // extern "C"
