// dr_internal.cuh -- internal declarations shared by the CUDA sources of the
// dynrecon library (plan layout, per-projection tables, launch helpers).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dynrecon.h"

namespace dr {

typedef __nv_bfloat16 bf16;

// ---------------------------------------------------------------------------
// Error reporting (thread-local message, status codes).
// ---------------------------------------------------------------------------
dr_status fail(dr_status st, const std::string &msg);
dr_status cuda_fail(cudaError_t e, const char *what);
void clear_error();

#define DR_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return dr::cuda_fail(_e, #expr); \
    } while (0)

// ---------------------------------------------------------------------------
// Device status word: kernels OR these bits in when a bounded wait gives up.
// ---------------------------------------------------------------------------
enum : int { kStatusTimeout = 1 };

// Template sizes for the number of basis functions: m is rounded up to the
// next supported M; tables are zero padded so the extra lanes add zeros.
int template_m(int m);

// ---------------------------------------------------------------------------
// Per-projection forward (Joseph) parameters.  For branch 0 the "lines" are
// image rows y_r and samples run along x; for branch 1 lines are columns x_r
// and samples run along y.  The sample position in pixel-index units along
// the line for bin b and line r is  xi = C + b*A + r*B.
// ---------------------------------------------------------------------------
struct FwdProj {
    long long A_fx, B_fx, C_fx;  // xi in 32.32 fixed point
    double A, B, C;              // xi in double (FP64 path)
    float Af, Bf, Cf;            // float copies for the loop-range estimate
    float scale;                 // 1/|cos| (branch 0) or 1/|sin| (branch 1)
    double scale_d;
    int branch;
    int pad_;
};

// Per-projection adjoint parameters: pos(i, j) = i*c + j*s + C0 is the ray
// coordinate of pixel (i, j) in bin-index units; cm = max(|c|, |s|).
struct AdjProj {
    double c, s, C0, inv_c;
};

// Adjoint tile shape: 8*VPT x 16 voxels, 128 threads, VPT voxels per thread.
constexpr int kAdjThreads = 128;
constexpr int kAdjTY = 16;
constexpr int kAdjP = 32;      // projections per pipeline stage
constexpr int kAdjStages = 3;  // TMA pipeline depth

constexpr int kFwdThreads = 256;
constexpr int kFwdRPT = 8;   // rays per thread
constexpr int kFwdGuard = 4; // zero cells on each side of a staged line
// Staged lines of the folded forward's strips: the even pixels of a line,
// then its odd pixels, each half with kFoldGuardE zero entries on both sides.
// A Joseph sample reads pixels i0 and i0 + 1, one even and one odd, so its
// two loads go to different halves; the eight lanes of a 16-byte load phase
// (consecutive bins, 1 to sqrt 2 pixels apart) then span at most 6 entries of
// a half and never share a bank slot (lanes on the same entry are served by
// one broadcast).  The odd half starts 4 slots (mod 8) after the even one, so
// the staging stores of neighbouring pixels do not collide either, and the
// line stride is odd, so stores of one pixel on consecutive lines (the
// column-stepping branch) do not.
constexpr int kFoldGuardE = 2;
__host__ __device__ constexpr int fold_half(int W) { return (W + 1) / 2 + 2 * kFoldGuardE; }
__host__ __device__ constexpr int fold_odd_off(int W) { return fold_half(W) + ((4 - fold_half(W)) & 7); }
__host__ __device__ constexpr int fold_line_elems(int W) { return (fold_odd_off(W) + fold_half(W)) | 1; }
// Strip lines staged by TMA (the static transforms of 4-float coefficient
// groups): each half of a line is written by copies of bw pixels taken every
// second pixel (a tensor map with element stride 2), bw/2 16-byte entries per
// copy at 128-byte aligned offsets; 8 zero entries before, between and after
// the halves.
__host__ __device__ constexpr int fold_tma_bw(int W) { return W >= 256 ? 256 : ((W + 15) / 16) * 16; }
__host__ __device__ constexpr int fold_tma_nbox(int W) { return (W + fold_tma_bw(W) - 1) / fold_tma_bw(W); }
__host__ __device__ constexpr int fold_tma_half(int W) { return fold_tma_nbox(W) * fold_tma_bw(W) / 2; }
__host__ __device__ constexpr int fold_tma_line(int W) { return 2 * fold_tma_half(W) + 24; }
constexpr int kFoldTmaStages = 2;  // TMA strip buffers (one CTA barrier per strip)
inline int fold_line_elems_max(int nx, int ny) {
    return fold_line_elems(nx) > fold_line_elems(ny) ? fold_line_elems(nx) : fold_line_elems(ny);
}
// Shared-memory budget of the folded forward's strip (float lines; both
// buffers when double-buffered): two CTAs of 256 threads still fit an SM.
constexpr int kFoldStripBudget = 110 * 1024;
constexpr int kFold2BlockVariants = 4;
// Static-transform CTA configurations of the two-kernel folded forward:
// MC = 4 or 8 coefficients (odd gi: 8); gi = 0..5: 256, 512 or 1024 threads
// (gi / 2), one CTA per SM at the larger sizes; gi = 6, 7: 512 threads with
// half the rays, two CTAs per SM (<= 64 registers), so that one CTA's strip
// barrier leaves the other running.
constexpr int kFold2Configs = 8;
__host__ __device__ constexpr int fold_static_mc(int gi) { return (gi & 1) ? 8 : 4; }
__host__ __device__ constexpr int fold_static_threads(int gi) { return gi < 6 ? 256 << (gi / 2) : 512; }
// rays per thread
__host__ __device__ constexpr int fold_static_rpt_gi(int gi) {
    return gi < 4 ? 32 / fold_static_mc(gi) : 16 / fold_static_mc(gi);
}
__host__ __device__ constexpr int fold_static_min_blocks(int gi) { return gi < 6 ? 1 : 2; }
__host__ __device__ constexpr int fold_static_rays(int gi) { return fold_static_threads(gi) * fold_static_rpt_gi(gi); }

constexpr int kRedThreads = 256;
constexpr int kRedBlocksMax = 1024;
constexpr int kRedSlots = 16;
constexpr int kRedSlotStride = 2 * kRedBlocksMax;  // doubles per slot (up to 2 values per block)

// Device-resident solver scalars (double).
struct DevScalars {
    double rr;      // <r, r>
    double pq;      // <p, A p>
    double alpha;   // CG step
    double beta;    // CG direction update
    double lam;     // power iteration: ||y||
    double acc0, acc1, acc2;
    int active;     // CG still running this u-step
    int iter;       // outer iteration counter (graph replay index)
    int pad_[2];
};

// Reduction slots (one per reducing kernel of an iteration).
enum RedSlot {
    kSlotRhs = 0,
    kSlotLap = 1,
    kSlotUpd = 2,
    kSlotFid = 3,
    kSlotProx = 4,
    kSlotPow = 5,
    kSlotTv = 6,
    kSlotDot = 7,
};

struct Workspace {
    size_t bytes = 0;
    dr_algo algo = DR_ADMM_CG;
    void *r = nullptr, *p = nullptr, *q = nullptr;  // [V][m] T
    void *ut = nullptr, *uold = nullptr;            // CP
    void *gd = nullptr;                             // data-sized scratch (S)
    void *h1 = nullptr;                             // CP dual, data sized (S)
    void *mu = nullptr, *w = nullptr;               // [nz][nt][ny][nx][4] field type
    void *u_dev = nullptr, *g_dev = nullptr;        // staging copies of host buffers
    double *obj = nullptr;                          // [iters][3] fid, tv, primal^2
    int obj_cap = 0;
};

}  // namespace dr

// The opaque plan.
struct dr_plan {
    int nx, ny, nz, ns, K, m, nt;
    // slab launches (slabs.cu): the TV stencils treat the slice below local
    // z = 0 / above local z = nz-1 as present; 0 for whole-volume launches
    int z_open_lo = 0, z_open_hi = 0;
    int M;   // template size >= m
    int MP;  // padded row length of the projection basis table (multiple of 4)
    int MT;  // TV template size >= m (4, 8, 16 or 32): row stride of the frame tables
    dr_basis basis;
    bool orthonormal = false;
    dr_precision prec;
    bool fields_bf16 = false;  // the solvers' dual fields stored in bf16 (DR_FIELDS_BF16)
    cudaStream_t stream;
    cudaStream_t graph_stream;
    cudaEvent_t ev_a, ev_b;
    int device;
    int num_sms;

    std::vector<double> theta, t, Phi, PhiF;  // host, double

    // device tables
    dr::FwdProj *d_fwd = nullptr;
    dr::AdjProj *d_adj = nullptr;
    void *d_PhiP = nullptr;      // [K][MP] T (zero padded)
    int *d_fwd_blocks = nullptr; // [n_fwd_blocks][fwd_P]
    int n_fwd_blocks = 0;
    int fwd_P = 0;
    int fwd_R = 0;
    void *d_PhiF = nullptr;   // [nt][MT] T
    void *d_dPhiF = nullptr;  // [nt][MT] T, row l = PhiF[l+1] - PhiF[l] (0 for the last)
    void *d_G = nullptr;      // [MT][MT] T, PhiF^T PhiF
    void *d_Lt = nullptr;     // [MT][MT] T, PhiF^T Lt PhiF (Lt = 1D Neumann Laplacian in l)
    std::vector<double> h_G, h_Lt;      // host copies of G and Lt ([MT][MT])
    std::vector<double> h_phif, h_dphif;  // host copies of PhiF and dPhiF ([nt][MT])
    // half-turn fold (Sec. 4): projections grouped by theta mod pi
    int fold_U = 0;                   // unique angles (0: the fold is unavailable for this plan)
    int fold_maxgrp = 0;              // largest group
    dr::FwdProj *d_fold_fwd = nullptr;  // [U] Joseph constants of the unique angles
    dr::AdjProj *d_fold_adj = nullptr;  // [U]
    int *d_fold_start = nullptr;      // [U+1] member ranges
    int *d_fold_member = nullptr;     // [K] 2*k + (1 if theta_k = theta0 + odd multiple of pi)
    int *d_fold_blocks = nullptr;     // [n_fold_blocks][fold_P] unique angles grouped by stepping axis
    int n_fold_blocks = 0, fold_P = 0, fold_R = 0, fold_nchunk = 1;
    int fold_lines = 0, fold_async = 0;  // folded forward: strip lines per buffer, cp.async double buffering
    int fold_lines_st = 0, fold_async_st = 0;  // the same for the bf16-strip kernel of BF16 plans
    bool fold_fwd_ok = false;         // the forward strip fits in shared memory
    // folded forward in two kernels (variant 2): static transforms of groups of
    // 4 or 8 coefficients of the distinct angles into d_gt, then distribution
    // configurations gi = 0..5: 4 / 8 coefficients (odd gi: 8) x 256 / 512 / 1024 threads (gi / 2)
    // angle blocks: variant v spreads each stepping axis's angles evenly over v more
    // blocks than the fewest that fit a CTA (smaller blocks, more CTAs: fuller last wave)
    int fold2_nchunk[dr::kFold2Configs] = {}, fold2_R[dr::kFold2Configs] = {};
    int fold2_Rt[dr::kFold2Configs] = {};  // strip lines of TMA staging (two buffers in twice the budget; 0: none)
    int fold2_P[dr::kFold2Configs][dr::kFold2BlockVariants] = {};
    int fold2_nblocks[dr::kFold2Configs][dr::kFold2BlockVariants] = {};
    int *d_fold2_blocks[dr::kFold2Configs][dr::kFold2BlockVariants] = {};
    int fold2_bv = 0;                 // angle-block variant in use
    bool fold2_ok = false;
    int fold2_gi = 0;                 // configuration in use
    int fold2_gi_st = 0;              // configuration of storage-typed (bf16-strip) calls of BF16 plans
    int sel_fwd_st = 0;               // forward variant of storage-typed calls on BF16 plans (bf16 strips)
    int fold2_split = 1;              // line chunks of the static march (partial sums added by the distribution)
    int fold2_async = 0, fold2_async_st = 0;  // double-buffered cp.async strips (compute-typed / bf16 kernels)
    int fold_adj_pp = 8;              // folded adjoint: distinct angles per pipeline stage
    void *d_fold_gram = nullptr;      // [U][M][M] float: sum over an angle's projections of phi phi^T
    bool split_off = false;           // set while a slab-streamed solve borrows the plan (its memory is budgeted)
    void *d_ru_split = nullptr;       // partial sums of a split march (allocated on first use)
    size_t ru_split_bytes = 0;
    int fold2_lines = 1, fold2_lines_st = 1;  // strip lines (compute-typed / bf16 kernels)
    void *d_gt = nullptr;             // folded data [nz][U][ns][MS] float (allocated on first use)
    size_t gt_bytes = 0;
    int var_fwd = -1, var_adj = -1;   // -1 automatic, 0 direct, 1 fold, 2 fold in two kernels (forward)
    int sel_fwd = 0, sel_adj = 0;     // variant in use
    bool tuned = false;
    double tune_ms[5] = {0, 0, 0, 0, 0}; // fwd direct, fwd fold, adj direct, adj fold, fwd fold (two kernels)
    double *d_partials = nullptr;
    unsigned *d_counters = nullptr;
    dr::DevScalars *d_scal = nullptr;
    int *d_status = nullptr;
    size_t table_bytes = 0;
    // FBP initial guess scratch (allocated on first use, fbp.cu)
    void *d_fbp_taps = nullptr;  // [2 ns - 1] T, Shepp-Logan taps
    void *d_fbp_phi = nullptr;   // [K][MP] T, window least-squares table used in place of PhiP
    void *d_fbp_q = nullptr;     // [nz][K][ns] T, filtered data
    void *d_fbp_u = nullptr;     // [V][m] float, result before BF16 rounding (BF16 plans)
    size_t fbp_bytes = 0;

    dr::Workspace ws;
    // set by the serving layer for its jobs: admm_solve stops between
    // iterations once the flag is raised (dr_server_cancel of a running job)
    const std::atomic<int> *cancel = nullptr;
};

namespace dr {

inline size_t elem_size(dr_precision p) { return p == DR_F64 ? 8 : (p == DR_BF16_F32ACC ? 2 : 4); }
inline size_t calc_size(dr_precision p) { return p == DR_F64 ? 8 : 4; }
// bytes per element of the solvers' dual fields
inline size_t field_size(const dr_plan *P) { return P->fields_bf16 ? 2 : calc_size(P->prec); }
inline size_t nvox(const dr_plan *P) { return (size_t)P->nx * P->ny * P->nz; }
inline size_t nu_elems(const dr_plan *P) { return nvox(P) * P->m; }
inline size_t ng_elems(const dr_plan *P) { return (size_t)P->nz * P->K * P->ns; }
inline size_t nf_elems(const dr_plan *P) { return nvox(P) * P->nt * 4; }

inline int red_grid(size_t n) {
    size_t b = (n + kRedThreads - 1) / kRedThreads;
    if (b < 1) b = 1;
    if (b > (size_t)kRedBlocksMax) b = kRedBlocksMax;
    return (int)b;
}

// Launchers (cudaStream_t = the stream to enqueue on).  Storage-typed
// pointers are void*; the plan's precision selects the instantiation.
//
// Forward projection epilogues: out = R u (mode 0), out = R u - gm (mode 1),
// out = (out + sigma R u - sigma gm) / (1 + sigma) (mode 2, CP dual h1).
dr_status launch_fwd(dr_plan *P, const void *u, void *out, const void *gm, int mode, double sigma,
                     cudaStream_t st);
// u = alpha R* g + beta u.  g and u are storage typed unless u_calc is set,
// in which case u is a compute-typed (float/double) vector.
dr_status launch_adj(dr_plan *P, const void *g, void *u, double alpha, double beta, bool u_calc,
                     cudaStream_t st);

// TV family (tv.cu).  "calc" pointers are compute typed, storage pointers S.
dr_status launch_grad(dr_plan *P, const void *u, bool u_calc, void *p, double lambda2, cudaStream_t st);
dr_status launch_grad_adj(dr_plan *P, const void *p, void *u, bool u_calc, double lambda2,
                          double alpha, double beta, cudaStream_t st);
dr_status launch_prox(dr_plan *P, const void *u, bool u_calc, void *mu, void *w, double rho,
                      double lambda1, double lambda2, double *obj_row, cudaStream_t st);
// out = beta*out + alpha * D^T D x, with <x, out> reduced into scal->pq and
// the CG step decided when cg_step is set.
dr_status launch_lap(dr_plan *P, const void *x, void *out, double alpha, double beta, double lambda2,
                     int cg_step, cudaStream_t st);
// r = r + rho (D^T w - D^T D u); p = r; scal->rr = <r, r>; scal->active = 1.
dr_status launch_rhs(dr_plan *P, const void *u, const void *w, void *r, void *p, double rho,
                     double lambda2, cudaStream_t st);
// h2 = project(h2 + sigma D ut, lambda1) (CP step 4).
dr_status launch_cp_dual(dr_plan *P, const void *ut, void *h2, double sigma, double lambda1,
                         double lambda2, cudaStream_t st);
// u_new = u - tau (a + D^T h2); ut = u_new + theta (u_new - u) (CP steps 5, 6).
dr_status launch_cp_primal(dr_plan *P, void *u, void *ut, const void *a, const void *h2, double tau,
                           double theta, double lambda2, cudaStream_t st);
// tv = sum |D u| into obj_row[1] (objective for CP).
dr_status launch_tv_sum(dr_plan *P, const void *u, double lambda2, double *obj_row, cudaStream_t st);

// Vector kernels (solver.cu).
dr_status launch_dot_to(dr_plan *P, const void *a, const void *b, size_t n, bool storage, double *dst,
                        cudaStream_t st);

// Allow `smem` bytes of dynamic shared memory for kernel `fn` on the current
// device.  The attribute is process-wide per kernel while plans on several
// threads launch it with different sizes, so it is raised once per kernel and
// device to the device's opt-in maximum (never set to one launch's size,
// which another thread could undercut between its set and its launch).
dr_status allow_dynamic_smem(const void *fn, size_t smem);

// Host-side tensor-map encoder (driver entry point, resolved once).
bool encode_tensor_map_2d(CUtensorMap *map, CUtensorMapDataType dt, void *base, uint64_t dim0,
                          uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1);
// rank-dimensional tiled map: dims[rank], strides[rank-1] (bytes, dims 1..), box[rank];
// elem_strides[rank] (nullptr: all 1): the box takes every k-th element of a
// dimension, box[i] / elem_strides[i] of them
bool encode_tensor_map(CUtensorMap *map, CUtensorMapDataType dt, int rank, void *base, const uint64_t *dims,
                       const uint64_t *strides, const uint32_t *box, const uint32_t *elem_strides = nullptr);

// Direct and folded projector variants; selection per plan (projector.cu).
dr_status launch_fwd_variant(dr_plan *P, int variant, bool calc, const void *u, void *out, const void *gm,
                             int mode, double sigma, cudaStream_t st);
dr_status launch_adj_variant(dr_plan *P, int variant, bool calc, const void *g, void *u, double alpha,
                             double beta, bool u_calc, cudaStream_t st);
dr_status ensure_fold_scratch(dr_plan *P);
dr_status ensure_split_scratch(dr_plan *P, size_t bytes);
// y = R*R x on compute-typed buffers; gscratch: a projection-sized buffer used
// when the folded normal operator does not apply
dr_status launch_normal_calc(dr_plan *P, const void *x, void *y, void *gscratch, cudaStream_t st);
// largest split scratch the autotuner may choose (small grids only need it)
constexpr size_t kSplitScratchMax = 256ull << 20;
dr_status autotune(dr_plan *P, void *u_scratch, void *g_scratch);

}  // namespace dr
