// fbp.cu -- filtered back-projection initial guess (Sec. 5 starts the
// iterations from an FBP reconstruction with the Shepp-Logan filter).
//
//   1. q[z][k][.] = h * g[z][k][.]   discrete Shepp-Logan kernel at unit bin
//      spacing, h(n) = -2 / (pi^2 (4 n^2 - 1)), linear (zero-padded)
//      convolution along s (shepp_logan_kernel below).
//   2. Projection k belongs to time window w(k) = clamp(floor(t_k nw)); the FBP
//      image of window w is f_w = (pi / K_w) sum_{k in w} R*_k q_k.  The
//      coefficients are the least-squares fit over the acquisition times,
//      u = argmin sum_k || sum_j phi_j(t_k) u_j - f_{w(k)} ||^2, i.e.
//      u_j = sum_w A[j][w] f_w with A = Phi^+ S (minimum-norm least squares,
//      (Phi^T Phi)^{-1} Phi^T S for functions independent over the times).
//      Both steps are linear in q, so u_j = sum_k Psi[k][j] R*_k q_k with
//      Psi[k][j] = (pi / K_{w(k)}) A[j][w(k)]: one dynamic back-projection
//      with the table Psi in place of Phi (either projector variant).
#include <algorithm>
#include <cmath>
#include <vector>

#include "dr_device.cuh"

namespace dr {

dr_status launch_adj_calc(dr_plan *P, const void *g, void *u, double alpha, double beta, cudaStream_t st);

constexpr int kFbpThreads = 256;

// One CTA filters whole rows (grid-stride over the nz*K rows).  Shared
// memory holds the taps h(n), n = -(ns-1)..ns-1, and the current row; the
// lanes of a warp read consecutive taps (no bank conflicts) and the same row
// element (broadcast).  Each output sums its row in ascending b'.
template <typename S, typename T>
__global__ void __launch_bounds__(kFbpThreads)
    shepp_logan_kernel(const S *__restrict__ g, T *__restrict__ q, const T *__restrict__ taps, long long rows,
                       int ns) {
    extern __shared__ __align__(16) unsigned char fbp_smem[];
    T *h = reinterpret_cast<T *>(fbp_smem);  // [2 ns - 1], h[i] = h(i - (ns - 1))
    T *row = h + (2 * ns - 1);                // [ns]
    const int nh = 2 * ns - 1;
    for (int i = threadIdx.x; i < nh; i += kFbpThreads) h[i] = taps[i];
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        __syncthreads();  // previous row consumed
        const S *gr = g + r * ns;
        for (int i = threadIdx.x; i < ns; i += kFbpThreads) row[i] = ldc<T>(gr + i);
        __syncthreads();
        for (int b = threadIdx.x; b < ns; b += kFbpThreads) {
            const T *hb = h + b + (ns - 1);  // hb[-b'] = h(b - b')
            T acc = T(0);
#pragma unroll 8
            for (int bp = 0; bp < ns; ++bp) acc = fma(hb[-bp], row[bp], acc);
            q[r * ns + b] = acc;
        }
    }
}

__global__ void fbp_to_bf16_kernel(const float *__restrict__ x, bf16 *__restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

template <typename S, typename T>
static dr_status launch_filter(dr_plan *P, const void *g, cudaStream_t st) {
    const long long rows = (long long)P->nz * P->K;
    const size_t smem = sizeof(T) * (size_t)(3 * P->ns - 1);
    auto kern = shepp_logan_kernel<S, T>;
    {
        dr_status s = allow_dynamic_smem((const void *)kern, smem);
        if (s != DR_OK) return s;
    }
    int per_sm = 0;
    DR_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFbpThreads, smem));
    const long long grid = std::min<long long>(rows, (long long)P->num_sms * std::max(per_sm, 1));
    kern<<<(unsigned)grid, kFbpThreads, smem, st>>>((const S *)g, (T *)P->d_fbp_q, (const T *)P->d_fbp_taps,
                                                    rows, P->ns);
    DR_CUDA_TRY(cudaGetLastError());
    return DR_OK;
}

template <typename T>
static dr_status upload_as(void *dst, const std::vector<double> &src) {
    std::vector<T> tmp(src.begin(), src.end());
    DR_CUDA_TRY(cudaMemcpy(dst, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice));
    return DR_OK;
}

// Eigen-decomposition of a symmetric n x n matrix by cyclic Jacobi rotations
// (Jacobi's method; Golub and Van Loan, Matrix Computations, Sec. 8.5):
// A = V diag(lam) V^T, V[i][e] = component i of eigenvector e.
static void sym_eig(std::vector<double> A, int n, std::vector<double> &V, std::vector<double> &lam) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            diag += A[(size_t)p * n + p] * A[(size_t)p * n + p];
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        }
        if (off <= 1e-32 * diag) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                const double th = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    lam.assign(n, 0.0);
    for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

// Psi[k][j] (row stride MP, zero padded) for nw windows.
static dr_status fbp_table(const dr_plan *P, int nw, std::vector<double> &psi) {
    const int K = P->K, m = P->m;
    std::vector<int> win(K);
    std::vector<long long> cnt(nw, 0);
    for (int k = 0; k < K; ++k) {
        const double x = std::floor(P->t[k] * nw);
        const int w = x < 0.0 ? 0 : (x > nw - 1 ? nw - 1 : (int)x);
        win[k] = w;
        ++cnt[w];
    }
    // Gram matrix Phi^T Phi = V diag(lam) V^T (cyclic Jacobi rotations)
    std::vector<double> G((size_t)m * m, 0.0), V, lam;
    for (int k = 0; k < K; ++k)
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) G[(size_t)i * m + j] += P->Phi[(size_t)k * m + i] * P->Phi[(size_t)k * m + j];
    sym_eig(G, m, V, lam);
    double lmax = 0.0;
    for (double l : lam) lmax = std::max(lmax, l);
    if (!(lmax > 0.0)) return fail(DR_EINVAL, "dr_fbp_init: the basis vanishes at every acquisition time");
    // A[:, w] = G^+ (sum_{k in w} Phi[k][:]): the minimum-norm least-squares
    // fit; eigenvalues below 1e-12 lam_max (singular values of Phi below
    // 1e-6 of the largest) count as zero
    std::vector<double> A((size_t)m * nw, 0.0), y(m);
    for (int w = 0; w < nw; ++w) {
        std::vector<double> rhs(m, 0.0);
        for (int k = 0; k < K; ++k)
            if (win[k] == w)
                for (int j = 0; j < m; ++j) rhs[j] += P->Phi[(size_t)k * m + j];
        for (int e = 0; e < m; ++e) {  // y = diag(1/lam) V^T rhs
            double v = 0.0;
            for (int j = 0; j < m; ++j) v += V[(size_t)j * m + e] * rhs[j];
            y[e] = lam[e] > 1e-12 * lmax ? v / lam[e] : 0.0;
        }
        for (int i = 0; i < m; ++i) {
            double v = 0.0;
            for (int e = 0; e < m; ++e) v += V[(size_t)i * m + e] * y[e];
            A[(size_t)i * nw + w] = v;
        }
    }
    psi.assign((size_t)K * P->MP, 0.0);
    for (int k = 0; k < K; ++k) {
        const int w = win[k];
        const double sc = M_PI / (double)cnt[w];
        for (int j = 0; j < m; ++j) psi[(size_t)k * P->MP + j] = sc * A[(size_t)j * nw + w];
    }
    return DR_OK;
}

static dr_status ensure(void **p, size_t bytes, size_t &acc) {
    if (*p) return DR_OK;
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "dr_fbp_init: scratch allocation");
    }
    acc += bytes;
    return DR_OK;
}

}  // namespace dr

using namespace dr;

extern "C" dr_status dr_fbp_init(dr_plan *P, const void *g, void *u, int n_windows) {
    clear_error();
    if (!P || !g || !u) return fail(DR_EINVAL, "dr_fbp_init: NULL argument");
    if (n_windows < 1 || n_windows > P->K) return fail(DR_EINVAL, "dr_fbp_init: n_windows must be in [1, K]");
    const size_t cs = calc_size(P->prec);
    const size_t ng = (size_t)P->nz * P->K * P->ns, nu = (size_t)P->nx * P->ny * P->nz * P->m;
    std::vector<double> psi;
    dr_status s = fbp_table(P, n_windows, psi);
    if (s != DR_OK) return s;

    // scratch (kept by the plan): taps, Psi, filtered data, FP32 result for BF16 plans
    const bool fresh_taps = P->d_fbp_taps == nullptr;
    if ((s = ensure(&P->d_fbp_taps, cs * (2 * (size_t)P->ns - 1), P->fbp_bytes)) != DR_OK) return s;
    if ((s = ensure(&P->d_fbp_phi, cs * (size_t)P->K * P->MP, P->fbp_bytes)) != DR_OK) return s;
    if ((s = ensure(&P->d_fbp_q, cs * ng, P->fbp_bytes)) != DR_OK) return s;
    if (P->prec == DR_BF16_F32ACC && (s = ensure(&P->d_fbp_u, sizeof(float) * nu, P->fbp_bytes)) != DR_OK) return s;

    // the tables may still be read by a previous call's kernels on this stream
    DR_CUDA_TRY(cudaStreamSynchronize(P->stream));
    if (fresh_taps) {
        std::vector<double> taps(2 * (size_t)P->ns - 1);
        for (int i = 0; i < 2 * P->ns - 1; ++i) {
            const double n = (double)(i - (P->ns - 1));
            taps[i] = -2.0 / (M_PI * M_PI * (4.0 * n * n - 1.0));
        }
        s = P->prec == DR_F64 ? upload_as<double>(P->d_fbp_taps, taps) : upload_as<float>(P->d_fbp_taps, taps);
        if (s != DR_OK) return s;
    }
    s = P->prec == DR_F64 ? upload_as<double>(P->d_fbp_phi, psi) : upload_as<float>(P->d_fbp_phi, psi);
    if (s != DR_OK) return s;

    cudaStream_t st = P->stream;
    switch (P->prec) {
        case DR_F32: s = launch_filter<float, float>(P, g, st); break;
        case DR_BF16_F32ACC: s = launch_filter<bf16, float>(P, g, st); break;
        case DR_F64: s = launch_filter<double, double>(P, g, st); break;
    }
    if (s != DR_OK) return s;

    // back-project with Psi in place of Phi (kernels take the table pointer at launch)
    void *phi = P->d_PhiP;
    P->d_PhiP = P->d_fbp_phi;
    if (P->prec == DR_BF16_F32ACC) s = launch_adj_calc(P, P->d_fbp_q, P->d_fbp_u, 1.0, 0.0, st);
    else s = launch_adj(P, P->d_fbp_q, u, 1.0, 0.0, false, st);
    P->d_PhiP = phi;
    if (s != DR_OK) return s;
    if (P->prec == DR_BF16_F32ACC) {
        const int grid = P->num_sms * 8;
        fbp_to_bf16_kernel<<<grid, 256, 0, st>>>((const float *)P->d_fbp_u, (bf16 *)u, nu);
        DR_CUDA_TRY(cudaGetLastError());
    }
    return DR_OK;
}
