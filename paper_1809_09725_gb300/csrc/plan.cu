// plan.cu -- plan construction (geometry and basis tables), error reporting,
// status handling and the tensor-map encoder of the dynrecon library.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "dr_device.cuh"
#include "dr_internal.cuh"

namespace dr {

static thread_local std::string g_last_error;

dr_status fail(dr_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

dr_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? DR_ENOMEM : DR_ECUDA;
}

void clear_error() { g_last_error.clear(); }

int template_m(int m) {
    static const int sizes[] = {1, 2, 4, 8, 12, 16, 24, 32};
    for (int s : sizes)
        if (m <= s) return s;
    return -1;
}

dr_status allow_dynamic_smem(const void *fn, size_t smem) {
    if (smem <= 48 * 1024) return DR_OK;
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> done;  // (kernel, device) -> allowed bytes
    int dev = 0;
    DR_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find({fn, dev});
    if (it == done.end()) {
        // the dynamic allowance is the opt-in maximum less the kernel's static shared memory
        int optin = 0;
        cudaFuncAttributes fa;
        cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
        const int limit = optin - (int)fa.sharedSizeBytes;
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
        if (e != cudaSuccess) {
            cudaGetLastError();  // not sticky: do not leave it for the next launch check
            return cuda_fail(e, "raising the dynamic shared-memory allowance");
        }
        it = done.emplace(std::make_pair(fn, dev), limit).first;
    }
    if (smem > (size_t)it->second)
        return fail(DR_EINVAL, "a kernel needs " + std::to_string(smem) + " bytes of shared memory, more than the device allows");
    return DR_OK;
}

// ---------------------------------------------------------------------------
// Temporal basis evaluation (Sec. 4, Eq. repr).  Real Fourier:
// phi_0 = 1, phi_{2i-1} = cos(2 pi i t), phi_{2i} = sin(2 pi i t).
// Shifted Legendre: phi_j(t) = P_j(2t - 1) by Bonnet's recurrence.  Haar,
// Heaviside steps, and the complex Fourier basis of Sec. 5 as real channel
// pairs (cos(w_j t), -sin(w_j t)), w_j = 2 pi (j - M/2).
// ---------------------------------------------------------------------------
static void eval_basis(dr_basis kind, int m, double t, double *row) {
    if (kind == DR_FOURIER_COMPLEX) {
        const int M = m / 2;
        for (int j = 0; j < M; ++j) {
            const double w = 2.0 * M_PI * (double)(j - M / 2);
            row[2 * j] = std::cos(w * t);
            row[2 * j + 1] = -std::sin(w * t);
        }
        return;
    }
    if (kind == DR_HAAR) {
        row[0] = 1.0;
        for (int j = 1; j < m; ++j) {
            int level = 31 - __builtin_clz((unsigned)j);  // j = 2^level + pos
            const int pos = j - (1 << level);
            const double x = std::ldexp(t, level) - pos;
            row[j] = (x >= 0.0 && x < 0.5) ? 1.0 : ((x >= 0.5 && x < 1.0) ? -1.0 : 0.0);
        }
        return;
    }
    if (kind == DR_HEAVISIDE) {
        row[0] = 1.0;
        for (int j = 1; j < m; ++j) row[j] = (t >= (double)j / (double)m) ? 1.0 : 0.0;
        return;
    }
    if (kind == DR_FOURIER_REAL) {
        row[0] = 1.0;
        for (int j = 1; j < m; ++j) {
            const int freq = (j + 1) / 2;
            const double a = 2.0 * M_PI * freq * t;
            row[j] = (j & 1) ? std::cos(a) : std::sin(a);
        }
    } else {
        const double x = 2.0 * t - 1.0;
        double pm1 = 1.0, p = x;
        row[0] = 1.0;
        if (m > 1) row[1] = x;
        for (int n = 1; n + 1 < m; ++n) {
            const double pn1 = ((2 * n + 1) * x * p - n * pm1) / (n + 1);
            row[n + 1] = pn1;
            pm1 = p;
            p = pn1;
        }
    }
}

static std::once_flag g_tmap_once;
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static void resolve_encoder() {
    std::call_once(g_tmap_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
}

bool encode_tensor_map(CUtensorMap *map, CUtensorMapDataType dt, int rank, void *base, const uint64_t *dims,
                       const uint64_t *strides, const uint32_t *box, const uint32_t *elem_strides) {
    resolve_encoder();
    if (!g_encode || rank < 1 || rank > 5) return false;
    cuuint64_t gdim[5], gstr[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        gdim[i] = dims[i];
        bx[i] = box[i];
        es[i] = elem_strides ? elem_strides[i] : 1;
        if (i + 1 < rank) gstr[i] = strides[i];
    }
    CUresult r = g_encode(map, dt, (cuuint32_t)rank, base, gdim, gstr, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_tensor_map_2d(CUtensorMap *map, CUtensorMapDataType dt, void *base, uint64_t dim0,
                          uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1) {
    resolve_encoder();
    if (!g_encode) return false;
    cuuint64_t gdim[2] = {dim0, dim1};
    cuuint64_t gstride[1] = {stride1_bytes};
    cuuint32_t box[2] = {box0, box1};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, dt, 2, base, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Adjoint constants of one angle: pixel (i, j) lies at bin position
// i*c + j*s + C0; the footprint half-width is max(|c|, |s|).
static AdjProj make_adj(double c, double s, double C0) {
    AdjProj a{};
    a.c = c;
    a.s = s;
    a.C0 = C0;
    a.inv_c = 1.0 / std::max(std::fabs(c), std::fabs(s));
    return a;
}

template <typename T>
static dr_status upload(void **dst, const std::vector<double> &src, size_t &bytes) {
    std::vector<T> tmp(src.size());
    for (size_t i = 0; i < src.size(); ++i) tmp[i] = (T)src[i];
    const size_t nb = std::max<size_t>(tmp.size(), 1) * sizeof(T);
    DR_CUDA_TRY(cudaMalloc(dst, nb));
    bytes += nb;
    if (!tmp.empty()) DR_CUDA_TRY(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
    return DR_OK;
}

static dr_status build_tables(dr_plan *P) {
    const int K = P->K, m = P->m, MP = P->MP, MT = P->MT, nt = P->nt;
    const bool dbl = P->prec == DR_F64;
    size_t &bytes = P->table_bytes;

    // basis at acquisition times and on the frame grid
    P->Phi.assign((size_t)K * m, 0.0);
    for (int k = 0; k < K; ++k) eval_basis(P->basis, m, P->t[k], &P->Phi[(size_t)k * m]);
    P->PhiF.assign((size_t)nt * m, 0.0);
    for (int l = 0; l < nt; ++l) eval_basis(P->basis, m, (double)l / nt, &P->PhiF[(size_t)l * m]);
    if (P->orthonormal) {
        // Gram matrix of the sampled functions, its Cholesky factor R (G = R^T R,
        // R upper with positive diagonal), then phi~ = phi R^{-1} for both tables.
        std::vector<double> G((size_t)m * m, 0.0), R((size_t)m * m, 0.0);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double a = 0.0;
                for (int k = 0; k < K; ++k) a += P->Phi[(size_t)k * m + i] * P->Phi[(size_t)k * m + j];
                G[(size_t)i * m + j] = a;
            }
        for (int j = 0; j < m; ++j) {
            double d = G[(size_t)j * m + j];
            for (int q = 0; q < j; ++q) d -= R[(size_t)q * m + j] * R[(size_t)q * m + j];
            if (!(d > 1e-24 * std::max(1.0, G[0]))) return fail(DR_EINVAL, "basis functions are dependent over the acquisition times");
            R[(size_t)j * m + j] = std::sqrt(d);
            for (int i = j + 1; i < m; ++i) {
                double e = G[(size_t)j * m + i];
                for (int q = 0; q < j; ++q) e -= R[(size_t)q * m + j] * R[(size_t)q * m + i];
                R[(size_t)j * m + i] = e / R[(size_t)j * m + j];
            }
        }
        auto apply = [&](std::vector<double> &tab, int rows) {
            for (int r = 0; r < rows; ++r) {
                double *row = &tab[(size_t)r * m];
                for (int j = 0; j < m; ++j) {  // solve x R = row (forward substitution over columns)
                    double v = row[j];
                    for (int q = 0; q < j; ++q) v -= row[q] * R[(size_t)q * m + j];
                    row[j] = v / R[(size_t)j * m + j];
                }
            }
        };
        apply(P->Phi, K);
        apply(P->PhiF, nt);
    }

    std::vector<double> phip((size_t)K * MP, 0.0);
    for (int k = 0; k < K; ++k)
        for (int j = 0; j < m; ++j) phip[(size_t)k * MP + j] = P->Phi[(size_t)k * m + j];
    std::vector<double> phif((size_t)nt * MT, 0.0), dphif((size_t)nt * MT, 0.0);
    for (int l = 0; l < nt; ++l)
        for (int j = 0; j < m; ++j) {
            phif[(size_t)l * MT + j] = P->PhiF[(size_t)l * m + j];
            if (l + 1 < nt)
                dphif[(size_t)l * MT + j] = P->PhiF[(size_t)(l + 1) * m + j] - P->PhiF[(size_t)l * m + j];
        }
    // G = PhiF^T PhiF ; Lt = PhiF^T Lt PhiF with (Lt F)_l = sum_{valid l' = l+-1} (F_l - F_l')
    std::vector<double> G((size_t)MT * MT, 0.0), Lt((size_t)MT * MT, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double g = 0.0, lt = 0.0;
            for (int l = 0; l < nt; ++l) {
                const double a = P->PhiF[(size_t)l * m + i];
                g += a * P->PhiF[(size_t)l * m + j];
                double lf = 0.0;
                if (l > 0) lf += P->PhiF[(size_t)l * m + j] - P->PhiF[(size_t)(l - 1) * m + j];
                if (l + 1 < nt) lf += P->PhiF[(size_t)l * m + j] - P->PhiF[(size_t)(l + 1) * m + j];
                lt += a * lf;
            }
            G[(size_t)i * MT + j] = g;
            Lt[(size_t)i * MT + j] = lt;
        }
    P->h_G = G;
    P->h_Lt = Lt;
    P->h_phif = phif;
    P->h_dphif = dphif;
    dr_status st;
    if (dbl) {
        if ((st = upload<double>(&P->d_PhiP, phip, bytes)) != DR_OK) return st;
        if ((st = upload<double>(&P->d_PhiF, phif, bytes)) != DR_OK) return st;
        if ((st = upload<double>(&P->d_dPhiF, dphif, bytes)) != DR_OK) return st;
        if ((st = upload<double>(&P->d_G, G, bytes)) != DR_OK) return st;
        if ((st = upload<double>(&P->d_Lt, Lt, bytes)) != DR_OK) return st;
    } else {
        if ((st = upload<float>(&P->d_PhiP, phip, bytes)) != DR_OK) return st;
        if ((st = upload<float>(&P->d_PhiF, phif, bytes)) != DR_OK) return st;
        if ((st = upload<float>(&P->d_dPhiF, dphif, bytes)) != DR_OK) return st;
        if ((st = upload<float>(&P->d_G, G, bytes)) != DR_OK) return st;
        if ((st = upload<float>(&P->d_Lt, Lt, bytes)) != DR_OK) return st;
    }

    // projection geometry
    const double hx = 0.5 * (P->nx - 1), hy = 0.5 * (P->ny - 1), hs = 0.5 * (P->ns - 1);
    std::vector<FwdProj> fw(K);
    std::vector<AdjProj> ad(K);
    std::vector<int> rows_b0, rows_b1;
    const double two32 = 4294967296.0;
    for (int k = 0; k < K; ++k) {
        const double c = std::cos(P->theta[k]), s = std::sin(P->theta[k]);
        FwdProj f{};
        if (std::fabs(c) >= std::fabs(s)) {
            f.branch = 0;
            f.A = 1.0 / c;
            f.B = -s / c;
            f.C = (-hs + hy * s) / c + hx;
            f.scale_d = 1.0 / std::fabs(c);
            rows_b0.push_back(k);
        } else {
            f.branch = 1;
            f.A = 1.0 / s;
            f.B = -c / s;
            f.C = (-hs + hx * c) / s + hy;
            f.scale_d = 1.0 / std::fabs(s);
            rows_b1.push_back(k);
        }
        f.A_fx = std::llround(f.A * two32);
        f.B_fx = std::llround(f.B * two32);
        f.C_fx = std::llround(f.C * two32);
        f.Af = (float)f.A;
        f.Bf = (float)f.B;
        f.Cf = (float)f.C;
        f.scale = (float)f.scale_d;
        fw[k] = f;
        ad[k] = make_adj(c, s, -hx * c - hy * s + hs);
    }
    DR_CUDA_TRY(cudaMalloc(&P->d_fwd, sizeof(FwdProj) * K));
    DR_CUDA_TRY(cudaMalloc(&P->d_adj, sizeof(AdjProj) * K));
    bytes += (sizeof(FwdProj) + sizeof(AdjProj)) * K;
    DR_CUDA_TRY(cudaMemcpy(P->d_fwd, fw.data(), sizeof(FwdProj) * K, cudaMemcpyHostToDevice));
    DR_CUDA_TRY(cudaMemcpy(P->d_adj, ad.data(), sizeof(AdjProj) * K, cudaMemcpyHostToDevice));

    // forward CTA work lists: blocks of fwd_P projections of one branch
    const int Pf = std::max(1, std::min(64, (kFwdThreads * kFwdRPT) / P->ns));
    P->fwd_P = Pf;
    const int Wmax = std::max(P->nx, P->ny);
    const int wpad = Wmax + 2 * kFwdGuard + 1;
    const size_t budget = 72 * 1024;
    int R = (int)(budget / ((size_t)Pf * wpad * calc_size(P->prec)));
    R = std::max(1, std::min(16, R));
    P->fwd_R = R;
    std::vector<int> blocks;
    for (const std::vector<int> *grp : {&rows_b0, &rows_b1}) {
        for (size_t i = 0; i < grp->size(); i += Pf) {
            for (int q = 0; q < Pf; ++q) {
                const size_t idx = i + q;
                blocks.push_back(idx < grp->size() ? (*grp)[idx] : -1);
            }
        }
    }
    P->n_fwd_blocks = (int)(blocks.size() / Pf);
    DR_CUDA_TRY(cudaMalloc(&P->d_fwd_blocks, sizeof(int) * std::max<size_t>(blocks.size(), 1)));
    bytes += sizeof(int) * blocks.size();
    if (!blocks.empty())
        DR_CUDA_TRY(cudaMemcpy(P->d_fwd_blocks, blocks.data(), sizeof(int) * blocks.size(), cudaMemcpyHostToDevice));

    // ---- half-turn fold (Sec. 4): group projections by theta mod pi ----
    if (P->prec != DR_F64) {
        struct Ent { double th0; int k, flip; };
        std::vector<Ent> ent(K);
        for (int k = 0; k < K; ++k) {
            const double n = std::floor(P->theta[k] / M_PI);
            double th0 = P->theta[k] - n * M_PI;
            long long ni = (long long)n;
            if (th0 >= M_PI) { th0 -= M_PI; ++ni; }
            if (th0 < 0.0) { th0 += M_PI; --ni; }
            ent[k] = Ent{th0, k, (int)(((ni % 2) + 2) % 2)};
        }
        std::sort(ent.begin(), ent.end(), [](const Ent &a, const Ent &b) {
            return a.th0 < b.th0 || (a.th0 == b.th0 && a.k < b.k);
        });
        // angles within 1e-11 rad of the group's first member share it; an angle
        // just below pi joins the group of 0 with the opposite parity
        const double tol = 1e-11;
        std::vector<int> start{0};
        std::vector<double> rep{ent.empty() ? 0.0 : ent[0].th0};
        for (int i = 1; i < K; ++i)
            if (ent[i].th0 - rep.back() > tol) {
                start.push_back(i);
                rep.push_back(ent[i].th0);
            }
        start.push_back(K);
        std::vector<int> member(K);
        for (int i = 0; i < K; ++i) member[i] = 2 * ent[i].k + ent[i].flip;
        if (rep.size() > 1 && M_PI - rep.back() <= tol) {
            // merge the last group into the first with flipped parity
            const int s0 = start[start.size() - 2];
            std::vector<int> merged;
            for (int i = s0; i < K; ++i) merged.push_back(member[i] ^ 1);
            std::vector<int> rest(member.begin(), member.begin() + s0);
            member.assign(merged.begin(), merged.end());
            member.insert(member.end(), rest.begin(), rest.end());
            const int shift = K - s0;
            std::vector<int> ns2{0};
            for (size_t g = 1; g + 1 < start.size() - 1; ++g) ns2.push_back(start[g] + shift);
            ns2.push_back(K);
            start = ns2;
            rep.pop_back();
        }
        const int U = (int)rep.size();
        int maxg = 0;
        for (int a = 0; a < U; ++a) maxg = std::max(maxg, start[a + 1] - start[a]);
        std::vector<FwdProj> ufw(U);
        std::vector<AdjProj> uad(U);
        std::vector<int> ub0, ub1;
        for (int a = 0; a < U; ++a) {
            const double c = std::cos(rep[a]), s = std::sin(rep[a]);
            FwdProj f{};
            if (std::fabs(c) >= std::fabs(s)) {
                f.branch = 0; f.A = 1.0 / c; f.B = -s / c; f.C = (-hs + hy * s) / c + hx; f.scale_d = 1.0 / std::fabs(c);
                ub0.push_back(a);
            } else {
                f.branch = 1; f.A = 1.0 / s; f.B = -c / s; f.C = (-hs + hx * c) / s + hy; f.scale_d = 1.0 / std::fabs(s);
                ub1.push_back(a);
            }
            f.A_fx = std::llround(f.A * two32); f.B_fx = std::llround(f.B * two32); f.C_fx = std::llround(f.C * two32);
            f.Af = (float)f.A; f.Bf = (float)f.B; f.Cf = (float)f.C; f.scale = (float)f.scale_d;
            ufw[a] = f;
            uad[a] = make_adj(c, s, -hx * c - hy * s + hs);
        }
        // forward work lists over unique angles
        const int M = P->M;
        const int rpt = M <= 4 ? 8 : 32 / M;  // rays per thread of the folded forward
        const int rays = 256 * rpt;            // 256-thread CTAs
        int Pf, nchunk;
        // a thread marches rpt bins of one angle: ceil(ns / rpt) threads per angle
        if (P->ns <= rays) { Pf = std::min(64, 256 / ((P->ns + rpt - 1) / rpt)); nchunk = 1; }
        else { Pf = 1; nchunk = (P->ns + rays - 1) / rays; }
        const int MS = M <= 4 ? 4 : ((M % 8 == 0) ? M + 4 : M);
        const size_t line = sizeof(float) * (size_t)fold_line_elems_max(P->nx, P->ny) * MS;
        int R = (int)((kFoldStripBudget) / line);
        if (R < 1 && line + 768 <= 200 * 1024) R = 1;
        R = std::min(R, 16);
        P->fold_fwd_ok = R >= 1;
        std::vector<int> fb;
        for (const std::vector<int> *grp : {&ub0, &ub1})
            for (size_t i = 0; i < grp->size(); i += Pf)
                for (int q = 0; q < Pf; ++q) fb.push_back(i + q < grp->size() ? (*grp)[i + q] : -1);
        P->fold_U = U;
        P->fold_maxgrp = maxg;
        P->fold_P = Pf;
        P->fold_R = std::max(R, 1);  // lines of one strip buffer that fit the shared-memory strip budget
        P->fold_lines = P->fold_R;   // in use (the autotuner may choose fewer)
        P->fold_async = 0;
        P->fold_lines_st = P->fold_R;
        P->fold_async_st = 0;
        P->fold_nchunk = nchunk;
        P->n_fold_blocks = (int)(fb.size() / Pf);
        DR_CUDA_TRY(cudaMalloc(&P->d_fold_fwd, sizeof(FwdProj) * U));
        DR_CUDA_TRY(cudaMalloc(&P->d_fold_adj, sizeof(AdjProj) * U));
        DR_CUDA_TRY(cudaMalloc(&P->d_fold_start, sizeof(int) * (U + 1)));
        DR_CUDA_TRY(cudaMalloc(&P->d_fold_member, sizeof(int) * K));
        DR_CUDA_TRY(cudaMalloc(&P->d_fold_blocks, sizeof(int) * std::max<size_t>(fb.size(), 1)));
        bytes += (sizeof(FwdProj) + sizeof(AdjProj) + sizeof(int)) * U + sizeof(int) * (K + 1 + fb.size());
        DR_CUDA_TRY(cudaMemcpy(P->d_fold_fwd, ufw.data(), sizeof(FwdProj) * U, cudaMemcpyHostToDevice));
        DR_CUDA_TRY(cudaMemcpy(P->d_fold_adj, uad.data(), sizeof(AdjProj) * U, cudaMemcpyHostToDevice));
        DR_CUDA_TRY(cudaMemcpy(P->d_fold_start, start.data(), sizeof(int) * (U + 1), cudaMemcpyHostToDevice));
        DR_CUDA_TRY(cudaMemcpy(P->d_fold_member, member.data(), sizeof(int) * K, cudaMemcpyHostToDevice));
        if (!fb.empty())
            DR_CUDA_TRY(cudaMemcpy(P->d_fold_blocks, fb.data(), sizeof(int) * fb.size(), cudaMemcpyHostToDevice));
        P->gt_bytes = sizeof(float) * (size_t)P->nz * U * P->ns * MS;
        // per distinct angle the Gram matrix of its projections' basis rows:
        // the folded normal operator R*R of the CG steps mixes by it
        {
            std::vector<float> gram((size_t)U * M * M, 0.0f);
            std::vector<double> acc((size_t)m * m);
            for (int a = 0; a < U; ++a) {
                std::fill(acc.begin(), acc.end(), 0.0);
                for (int i = start[a]; i < start[a + 1]; ++i) {
                    const double *ph = &P->Phi[(size_t)(member[i] >> 1) * m];
                    for (int q = 0; q < m; ++q)
                        for (int j = 0; j < m; ++j) acc[(size_t)q * m + j] += ph[q] * ph[j];
                }
                for (int q = 0; q < m; ++q)
                    for (int j = 0; j < m; ++j) gram[((size_t)a * M + q) * M + j] = (float)acc[(size_t)q * m + j];
            }
            DR_CUDA_TRY(cudaMalloc(&P->d_fold_gram, sizeof(float) * gram.size()));
            DR_CUDA_TRY(cudaMemcpy(P->d_fold_gram, gram.data(), sizeof(float) * gram.size(), cudaMemcpyHostToDevice));
            bytes += sizeof(float) * gram.size();
        }
        // two-kernel folded forward: work lists and strip budgets of the
        // coefficient-group / CTA-shape configurations
        for (int gi = 0; gi < kFold2Configs; ++gi) {
            const int MC = fold_static_mc(gi);
            const int rays2 = fold_static_rays(gi);
            int Pmax, nch2;
            const int tpa2 = (P->ns + fold_static_rpt_gi(gi) - 1) / fold_static_rpt_gi(gi);
            if (P->ns <= rays2) { Pmax = std::min(64, fold_static_threads(gi) / tpa2); nch2 = 1; }
            else { Pmax = 1; nch2 = (P->ns + rays2 - 1) / rays2; }
            const int ps2 = MC == 4 ? 4 : 12;  // float strip stride of the group
            const size_t line2 = sizeof(float) * (size_t)fold_line_elems_max(P->nx, P->ny) * ps2;
            P->fold2_R[gi] = std::min(16, (int)(kFoldStripBudget / line2));
            // TMA strips (float data, m a multiple of 4): MC / 4 planes of 16-byte entries per pixel
            const size_t line_t = 16 * (size_t)(MC / 4) * std::max(fold_tma_line(P->nx), fold_tma_line(P->ny));
            P->fold2_Rt[gi] = (P->prec != DR_F64 && P->m % 4 == 0)
                                  ? std::min(16, (int)((2 * (size_t)kFoldStripBudget) / (kFoldTmaStages * line_t)))
                                  : 0;
            P->fold2_nchunk[gi] = nch2;
            const int nmax = (int)std::max(ub0.size(), ub1.size());
            for (int v = 0; v < kFold2BlockVariants; ++v) {
                // v more blocks per stepping axis than the fewest, angles spread evenly
                const int nb = (nmax + Pmax - 1) / Pmax + v;
                const int P2 = v == 0 ? Pmax : std::max(1, (nmax + nb - 1) / nb);
                if (v > 0 && (nch2 > 1 || P2 == P->fold2_P[gi][v - 1])) break;  // nothing new
                std::vector<int> fb2;
                for (const std::vector<int> *grp : {&ub0, &ub1})
                    for (size_t i = 0; i < grp->size(); i += P2)
                        for (int q = 0; q < P2; ++q) fb2.push_back(i + q < grp->size() ? (*grp)[i + q] : -1);
                P->fold2_P[gi][v] = P2;
                P->fold2_nblocks[gi][v] = (int)(fb2.size() / P2);
                DR_CUDA_TRY(cudaMalloc(&P->d_fold2_blocks[gi][v], sizeof(int) * std::max<size_t>(fb2.size(), 1)));
                if (!fb2.empty())
                    DR_CUDA_TRY(cudaMemcpy(P->d_fold2_blocks[gi][v], fb2.data(), sizeof(int) * fb2.size(),
                                           cudaMemcpyHostToDevice));
                bytes += sizeof(int) * fb2.size();
            }
        }
        P->fold2_ok = P->m >= 4 && P->fold2_R[0] >= 1;
        // default: groups of 4 coefficients, 256 threads (the autotuner times all)
        P->fold2_gi = P->fold2_gi_st = 0;
        P->fold2_lines = P->fold2_lines_st = std::max(1, std::min(4, P->fold2_R[0]));
        // cost model until measured: fold when the unique angles carry the work
        const double direct = (double)K * (P->m + 16), fold = (double)U * (3.0 * P->m + 12) + 0.05 * K * P->m;
        P->sel_fwd = (P->fold_fwd_ok && fold < 0.8 * direct) ? 1 : 0;
        P->sel_fwd_st = P->sel_fwd;
        P->sel_adj = (fold < 0.8 * direct) ? 1 : 0;
    }

    // reductions, scalars, status
    DR_CUDA_TRY(cudaMalloc(&P->d_partials, sizeof(double) * kRedSlots * kRedSlotStride));
    DR_CUDA_TRY(cudaMalloc(&P->d_counters, sizeof(unsigned) * kRedSlots));
    DR_CUDA_TRY(cudaMalloc(&P->d_scal, sizeof(DevScalars)));
    DR_CUDA_TRY(cudaMalloc(&P->d_status, sizeof(int)));
    bytes += sizeof(double) * kRedSlots * kRedSlotStride + sizeof(unsigned) * kRedSlots + sizeof(DevScalars) +
             sizeof(int);
    DR_CUDA_TRY(cudaMemset(P->d_counters, 0, sizeof(unsigned) * kRedSlots));
    DR_CUDA_TRY(cudaMemset(P->d_scal, 0, sizeof(DevScalars)));
    DR_CUDA_TRY(cudaMemset(P->d_status, 0, sizeof(int)));
    return DR_OK;
}

void free_workspace(dr_plan *P);

}  // namespace dr

using namespace dr;

extern "C" {

const char *dr_last_error(void) { return g_last_error.c_str(); }

const char *dr_version(void) { return "dynrecon 0.1 (sm_103a)"; }

void dr_solve_params_default(dr_solve_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->algo = DR_ADMM_CG;
    p->iters = 20;
    p->n_cg = 4;
    p->lambda1 = 1e-3;
    p->lambda2 = 1.0;
    p->rho = 0.0;
    p->cp_theta = 1.0;
    p->power_iters = 100;
}

dr_status dr_plan_create(dr_plan **out, int nx, int ny, int nz, int ns, int K, const double *theta,
                         const double *t, dr_basis basis, int m, int nt_frames, dr_precision prec,
                         void *cuda_stream) {
    clear_error();
    if (!out) return fail(DR_EINVAL, "dr_plan_create: out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || ns < 1 || K < 1 || nt_frames < 1)
        return fail(DR_EINVAL, "dr_plan_create: sizes must be >= 1");
    if (ns > 2048) return fail(DR_EINVAL, "dr_plan_create: ns > 2048 is not supported");
    if (nt_frames > 256) return fail(DR_EINVAL, "dr_plan_create: nt_frames > 256 is not supported");
    if (nx > 65536 || ny > 65536 || nz > 65535 || K > (1 << 24))
        return fail(DR_EINVAL, "dr_plan_create: size out of range");
    if (m < 1 || m > 32) return fail(DR_EINVAL, "dr_plan_create: m must be in [1, 32]");
    const int kind = (int)basis & 0xff, flags = (int)basis & ~0xff;
    if (kind < DR_FOURIER_REAL || kind > DR_FOURIER_COMPLEX || (flags & ~DR_BASIS_ORTHONORMAL))
        return fail(DR_EINVAL, "dr_plan_create: bad basis");
    if (kind == DR_FOURIER_COMPLEX && m % 2 != 0)
        return fail(DR_EINVAL, "dr_plan_create: the complex Fourier basis needs an even m (2 real channels per function)");
    const bool fields_bf16 = ((int)prec & DR_FIELDS_BF16) != 0;
    prec = (dr_precision)((int)prec & ~DR_FIELDS_BF16);
    if (prec != DR_F32 && prec != DR_BF16_F32ACC && prec != DR_F64)
        return fail(DR_EINVAL, "dr_plan_create: bad precision");
    if (fields_bf16 && prec == DR_F64)
        return fail(DR_EINVAL, "dr_plan_create: DR_FIELDS_BF16 needs a DR_F32 or DR_BF16_F32ACC plan");
    if (!theta || !t) return fail(DR_EINVAL, "dr_plan_create: theta/t are NULL");
    for (int k = 0; k < K; ++k)
        if (!std::isfinite(theta[k]) || !std::isfinite(t[k]))
            return fail(DR_EINVAL, "dr_plan_create: theta/t must be finite");

    dr_plan *P = new (std::nothrow) dr_plan();
    if (!P) return fail(DR_ENOMEM, "dr_plan_create: host allocation failed");
    P->nx = nx; P->ny = ny; P->nz = nz; P->ns = ns; P->K = K; P->m = m; P->nt = nt_frames;
    P->M = template_m(m);
    P->MP = (P->M + 3) / 4 * 4;
    P->MT = m <= 4 ? 4 : (m <= 8 ? 8 : (m <= 16 ? 16 : 32));
    P->basis = (dr_basis)kind;
    P->orthonormal = (flags & DR_BASIS_ORTHONORMAL) != 0;
    P->prec = prec;
    P->fields_bf16 = fields_bf16;
    P->stream = (cudaStream_t)cuda_stream;
    P->theta.assign(theta, theta + K);
    P->t.assign(t, t + K);
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P->graph_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->ev_b, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        dr_status st = cuda_fail(e, "dr_plan_create");
        dr_plan_destroy(P);
        return st;
    }
    dr_status st = build_tables(P);
    if (st != DR_OK) {
        std::string msg = g_last_error;
        dr_plan_destroy(P);
        return fail(st, msg);
    }
    *out = P;
    return DR_OK;
}

dr_status dr_plan_destroy(dr_plan *P) {
    if (!P) return DR_OK;
    // the plan's own streams only: a device-wide synchronisation would also
    // touch (and could invalidate) graph captures of other threads' plans
    cudaStreamSynchronize(P->stream);  // the caller's stream (0: the legacy stream)
    if (P->graph_stream) cudaStreamSynchronize(P->graph_stream);
    free_workspace(P);
    void *ptrs[] = {P->d_fwd,        P->d_adj,       P->d_PhiP,       P->d_fwd_blocks,  P->d_PhiF,
                    P->d_dPhiF,      P->d_G,         P->d_Lt,         P->d_partials,    P->d_counters,
                    P->d_scal,       P->d_status,    P->d_fold_fwd,   P->d_fold_adj,    P->d_fold_start,
                    P->d_fold_member, P->d_fold_blocks, P->d_gt, P->d_fbp_taps, P->d_fbp_phi, P->d_fbp_q,
                    P->d_fbp_u, P->d_ru_split, P->d_fold_gram};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &row : P->d_fold2_blocks)
        for (int *p : row)
            if (p) cudaFree(p);
    if (P->graph_stream) cudaStreamDestroy(P->graph_stream);
    if (P->ev_a) cudaEventDestroy(P->ev_a);
    if (P->ev_b) cudaEventDestroy(P->ev_b);
    delete P;
    return DR_OK;
}

dr_status dr_plan_set_stream(dr_plan *P, void *s) {
    if (!P) return fail(DR_EINVAL, "dr_plan_set_stream: NULL plan");
    P->stream = (cudaStream_t)s;
    return DR_OK;
}

size_t dr_plan_device_bytes(const dr_plan *P) {
    return P ? P->table_bytes + P->ws.bytes + (P->d_gt ? P->gt_bytes : 0) + P->fbp_bytes + P->ru_split_bytes : 0;
}

}  // extern "C"

namespace dr {
// Failure-path check of the bounded waits: an mbarrier that nothing arrives
// at, waited on with the same bounded wait the TMA pipelines use.  Every
// thread gives up after limit_ns, sets the status word and returns.
__global__ void wait_selftest_kernel(int *status, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    mbar_wait_bounded(&bar, 0u, status, limit_ns);
}
}  // namespace dr

extern "C" {

dr_status dr_plan_wait_selftest(dr_plan *P, double limit_s) {
    clear_error();
    if (!P) return fail(DR_EINVAL, "dr_plan_wait_selftest: NULL plan");
    if (!(limit_s > 0.0 && limit_s <= 2.0)) return fail(DR_EINVAL, "dr_plan_wait_selftest: limit_s must be in (0, 2]");
    dr::wait_selftest_kernel<<<1, 32, 0, P->stream>>>(P->d_status, (unsigned long long)(limit_s * 1e9));
    DR_CUDA_TRY(cudaGetLastError());
    return dr_plan_sync(P);
}

dr_status dr_plan_sync(dr_plan *P) {
    if (!P) return fail(DR_EINVAL, "dr_plan_sync: NULL plan");
    DR_CUDA_TRY(cudaStreamSynchronize(P->stream));
    DR_CUDA_TRY(cudaStreamSynchronize(P->graph_stream));
    DR_CUDA_TRY(cudaGetLastError());
    int flag = 0;
    DR_CUDA_TRY(cudaMemcpy(&flag, P->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        DR_CUDA_TRY(cudaMemset(P->d_status, 0, sizeof(int)));
        return fail(DR_ETIMEOUT, "a bounded device-side wait gave up (status word set)");
    }
    return DR_OK;
}

}  // extern "C"
