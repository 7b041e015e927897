/*
 * dynrecon.h -- C ABI of the GB300 (sm_103a) library for four-dimensional
 * tomographic reconstruction by time-domain decomposition (Nikitin,
 * Carlsson, Andersson, Mokso, arXiv 1809.09725).
 *
 * The object f(x, y, z, t) is represented by m temporal-basis coefficient
 * volumes u_j (Sec. 4, Eq. repr):  f(x, t) = sum_j phi_j(t) u_j(x).
 * Projection k is acquired at angle theta_k and time t_k under continuous
 * rotation (Sec. 2, Eq. Rfwd).  The regularised model is Eq. (lr12):
 *     min_u  1/2 || R u - g ||^2 + lambda1 sum_{x,l} | nabla_{lambda2} f(x, t_l) |
 * with the isotropic 4D gradient of Eq. (TV1) on nt reconstruction frames
 * t_l = l / nt (Sec. 4, Eq. discrt).
 *
 * Discretisation (the paper leaves it open; this is the library's):
 *   pixel centres  x_i = i - (nx-1)/2, y_j = j - (ny-1)/2 (unit pixels),
 *   detector bins  s_b = b - (ns-1)/2 (unit spacing), slices independent;
 *   R is the Joseph ray-driven projector (linear interpolation along the
 *   axis closer to the ray, weighted 1/max(|cos|,|sin|)); R* is its exact
 *   transpose; nabla uses forward differences with zero difference across
 *   the last index of each dimension, lambda2 scaling the time component.
 *
 * Layouts (row-major, last index fastest; all arrays dense):
 *   u    [nz][ny][nx][m]      coefficient volumes
 *   g    [nz][K][ns]          projection data
 *   p,mu,w [nz][nt][ny][nx][4] 4-vector fields on frames, frame-major
 *        within each slice (components d/dx, d/dy, d/dz, lambda2 d/dt)
 * Element type is set by the plan's precision:
 *   DR_F32          u, g, fields: float
 *   DR_BF16_F32ACC  u, g: bfloat16 (raw 16-bit); fields: float; all
 *                   arithmetic in float, inner products in double
 *   | DR_FIELDS_BF16 the solvers' own dual fields in bfloat16 (see below)
 *   DR_F64          everything double
 *
 * Memory and execution: unless a call says otherwise, data pointers are
 * DEVICE pointers owned by the caller, and calls are asynchronous on the
 * plan's stream.  The plan owns its tables and solver workspace.  No call
 * throws; every call returns a dr_status and, on failure, records a message
 * readable with dr_last_error() on the calling thread.
 */
#ifndef DYNRECON_H
#define DYNRECON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DR_OK = 0,
    DR_EINVAL = -1,     /* bad shape, pointer, parameter or unsupported size */
    DR_ENOMEM = -2,     /* device allocation failed or memory budget exceeded */
    DR_ECUDA = -3,      /* a CUDA runtime call failed */
    DR_ETIMEOUT = -4,   /* a bounded device-side wait gave up (status flag set) */
    DR_ENOTCONV = -5,   /* reserved: solver reported non-convergence */
    DR_ECANCELED = -6   /* a job was cancelled */
} dr_status;

typedef enum {
    DR_FOURIER_REAL = 0, /* phi_0 = 1, phi_{2i-1} = cos(2 pi i t), phi_{2i} = sin(2 pi i t) */
    DR_LEGENDRE = 1,     /* phi_j(t) = P_j(2t - 1), Legendre polynomials, unnormalised */
    DR_HAAR = 2,         /* phi_0 = 1; j = 2^l + p: +1 on [p, p+1/2)/2^l, -1 on [p+1/2, p+1)/2^l (Sec. 8) */
    DR_HEAVISIDE = 3,    /* phi_0 = 1, phi_j(t) = 1 for t >= j/m, else 0 (Sec. 4) */
    /* Complex Fourier basis of Sec. 5, phi_j(t) = exp(2 pi i t (j - M/2)),
     * j = 0..M-1 (M/2 rounded down), carried as m = 2M real channels: channel
     * 2j holds Re u_j with function cos(w_j t), channel 2j+1 holds Im u_j with
     * -sin(w_j t), w_j = 2 pi (j - M/2), so the object is Re sum_j u_j phi_j(t)
     * and the adjoint weights are conj(phi_j) as in Eq. (radadjapr).  m must
     * be even.  As a real basis it is redundant (cos(-w t) = cos(w t), sin 0 =
     * 0), so DR_BASIS_ORTHONORMAL rejects it. */
    DR_FOURIER_COMPLEX = 4,
    /* Flag OR-ed into the kind: orthonormalise the basis over the acquisition
     * times (Gram-Schmidt, Sec. 4): phi~ = phi R^{-1} with sum_k phi~_i(t_k)
     * phi~_j(t_k) = delta_ij; the frames use the same transformed functions. */
    DR_BASIS_ORTHONORMAL = 0x100
} dr_basis;

typedef enum {
    DR_F32 = 0,
    DR_BF16_F32ACC = 1,
    DR_F64 = 2,
    /* Flag OR-ed into DR_F32 or DR_BF16_F32ACC: the solvers (admm_solve,
     * admm_solve_batch, the serving layer) keep their dual fields -- ADMM's mu
     * and w, Chambolle-Pock's h2, 4 nt values per voxel, the largest part of
     * the solver state -- in bfloat16, each value rounded once to nearest on
     * every store, arithmetic in float.  Halves the fields' device memory and
     * HBM traffic; the operator entry points and the state buffer (resume)
     * are unchanged in layout, the state holding the fields as bf16.  The
     * slab-streamed solver keeps float fields.  Rejected for DR_F64. */
    DR_FIELDS_BF16 = 0x10
} dr_precision;

typedef enum {
    DR_ADMM_CG = 0,        /* ADMM split psi = D u, u-step by n_cg conjugate-gradient steps */
    DR_CHAMBOLLE_POCK = 1  /* primal-dual iteration of Sec. 3, Fig. 2 */
} dr_algo;

typedef struct dr_plan dr_plan;

/*
 * Create a plan for one reconstruction geometry (Sec. 4, Eq. discrt).
 *   nx, ny, nz  volume size (pixels per row, rows, slices), each >= 1
 *   ns          detector bins per projection row, 1 <= ns <= 2048
 *   K           number of projections, >= 1
 *   theta       host [K] projection angles in radians (any real value)
 *   t           host [K] acquisition times in [0, 1) (scan-normalised)
 *   basis, m    temporal basis kind (optionally | DR_BASIS_ORTHONORMAL) and size,
 *               1 <= m <= 32 (Sec. 4, Eq. repr); DR_EINVAL if orthonormalisation
 *               finds the functions dependent over the acquisition times
 *   nt_frames   number of reconstruction frames for the time derivative (<= 256),
 *               frame l at t = l / nt_frames, >= 1
 *   prec        storage/arithmetic precision (see above)
 *   cuda_stream cudaStream_t on which calls are issued (NULL = default stream)
 * Copies theta and t; allocates device tables.  Returns DR_EINVAL for bad
 * arguments, DR_ENOMEM / DR_ECUDA on allocation or runtime failure; *out is
 * left NULL on failure.  The current CUDA device at creation is the plan's.
 */
dr_status dr_plan_create(dr_plan **out, int nx, int ny, int nz, int ns, int K,
                         const double *theta, const double *t, dr_basis basis, int m,
                         int nt_frames, dr_precision prec, void *cuda_stream);

/* Release the plan and everything it owns (synchronises its stream).  NULL is a no-op. */
dr_status dr_plan_destroy(dr_plan *plan);

/* Change the stream later calls are issued on. */
dr_status dr_plan_set_stream(dr_plan *plan, void *cuda_stream);

/* Bytes of device memory the plan holds now (tables plus solver workspace). */
size_t dr_plan_device_bytes(const dr_plan *plan);

/* Bytes of solver workspace admm_solve would allocate for this plan and algo. */
size_t dr_plan_workspace_bytes(const dr_plan *plan, dr_algo algo);

/*
 * Projector variants.  0 = direct: every projection uses its own angle
 * (Eqs. radapr / radadjapr as written).  1 = half-turn fold (Sec. 4): with
 * theta_k = n_k pi + theta0_k, R f(theta_k, s) = R f(theta0_k, (-1)^n_k s), so
 * the static transform of each coefficient volume is computed once per
 * distinct theta0 (angles equal within 1e-11 rad) and distributed with the
 * weights phi_j(t_k); the adjoint first folds the data per theta0
 *     gt_j(theta0, s) = sum_{k: theta0_k = theta0} phi_j(t_k) g_k((-1)^n_k s)
 * and back-projects the m folded sinograms.  Same operator up to rounding;
 * the fold is offered for F32 and BF16 plans.  2 (forward only, m >= 4) =
 * the fold in two kernels: the static transforms of groups of 4 or 8
 * coefficients are computed by separate CTAs (more rays per staged image,
 * which pays off for wide images and large m) into the plan's folded-data
 * scratch, then distributed to the K projections.  -1 = automatic (a cost
 * model until dr_plan_autotune or admm_solve has timed them).  Returns
 * DR_EINVAL if a fold variant is requested but unavailable.
 */
dr_status dr_plan_set_variant(dr_plan *plan, int fwd_variant, int adj_variant);

/*
 * Time the variants of both projectors on this plan's geometry (allocates
 * and frees scratch; synchronises) and keep the fastest for automatic
 * selection; for the folded forwards also choose the strip height, staging
 * mode and coefficient group size (none changes the result).  The decision
 * is cached for the process, keyed by the sizes, basis, precision, angles and
 * times, so later plans of the same problem reuse it (same kernels,
 * bit-identical results) without timing again.  times_ms: HOST [5] nullable:
 * forward direct, forward fold, adjoint direct, adjoint fold, forward fold in
 * two kernels (-1 where a variant is unavailable).
 */
dr_status dr_plan_autotune(dr_plan *plan, double *times_ms);

/*
 * Fix the folded forward's strip: `lines` image lines staged in shared memory
 * per step (1 <= lines; lines (x 2 with async) within the plan's 110 KB strip
 * budget) and async = 1 for cp.async double buffering (F32 plans with m a
 * multiple of 4, BF16 plans with m a multiple of 8).  Every choice marches
 * each ray over the same lines in the same order, so results are identical;
 * only the time changes.  A later autotune may replace the choice.  DR_EINVAL
 * if the fold is unavailable or the choice does not fit.
 */
dr_status dr_plan_set_fold_strip(dr_plan *plan, int lines, int async);

/*
 * Fix the two-kernel folded forward's configuration: coefficients per CTA
 * (group 4, or 8 when m > 4), CTA size and rays per thread, and strip height
 * (lines >= 1, within the strip budget).  The configurations: threads 256 or
 * 512 with 32 / group rays per thread, 1024 with 16 / group (one CTA per SM at
 * 512 and 1024), and 512 with 16 / group (two CTAs per SM).  rays_per_thread
 * 0 picks the most rays per thread for the group and CTA size.  Every
 * coefficient's ray sums run the same march whatever the choice: results are
 * identical.  DR_EINVAL if the variant is unavailable or the choice does not
 * exist or fit.
 */
dr_status dr_plan_set_fold_groups(dr_plan *plan, int group, int threads, int rays_per_thread, int lines);

/*
 * Fix how the two-kernel folded forward marches its rays.  nsplit (1..8):
 * chunks of image lines per ray, nsplit times as many CTAs, each summing its
 * chunk; the distribution kernel adds the chunks' partial sums in chunk order
 * before the basis weights (Sec. 4 fold, Eq. 5 combine), so results change
 * only by the rounding of those additions.  nsplit > 1 costs nsplit * nz * U
 * * ns * ceil(m / 4) * 4 floats of device memory, allocated on the next
 * forward (call that outside graph capture); slab-streamed solves use one
 * chunk.  async 0: synchronous strip staging; 1: double-buffered strips, the
 * next copied with cp.async while the current is marched; 2: three buffers,
 * two strips ahead, one CTA barrier per strip (strips limited to twice the
 * strip budget; where one line does not fit three times, two buffers); 3:
 * strips copied by TMA (cp.async.bulk.tensor, even and odd pixels of a line
 * taken by tensor maps with element stride 2) into two buffers completing
 * on mbarriers, one CTA barrier per strip -- for 4-coefficient groups of
 * float data whose m is a multiple of 4, otherwise mode 2.  Same arithmetic in
 * every mode: results identical.
 * DR_EINVAL if the variant is unavailable or an argument is out of range.
 */
dr_status dr_plan_set_fold_march(dr_plan *plan, int nsplit, int async);

/*
 * Fix the folded adjoint's distinct angles per pipeline stage (1..32; the
 * autotuner picks among 8, 7 and 6).  Each stage's folded-data windows share
 * a CTA's shared memory, so fewer angles per stage fit more CTAs on an SM.
 * The angles are summed in the same order whatever the choice: results are
 * identical.  DR_EINVAL if the plan has no folded adjoint or angles is out of
 * range.
 */
dr_status dr_plan_set_fold_adj_stage(dr_plan *plan, int angles);

/*
 * Fix the two-kernel folded forward's angle blocks: extra (0..3) more blocks
 * per stepping axis than the fewest whose rays fill a CTA, with the angles
 * spread evenly over them (smaller blocks, more CTAs: a fuller last wave).
 * Each ray's march is unchanged: results are identical.
 * dr_plan_set_fold_groups resets it to 0: set it afterwards.
 * DR_EINVAL if the variant is unavailable or does not exist for this plan
 * (variants that would repeat the block size of the one below are not built).
 */
dr_status dr_plan_set_fold_blocks(dr_plan *plan, int extra);


typedef struct {
    int unique_angles;   /* distinct theta mod pi (0: the fold is unavailable) */
    int max_group;       /* most projections sharing one theta mod pi */
    int fwd_variant;     /* variant the forward uses now (0 direct, 1 fold, 2 fold in two kernels) */
    int adj_variant;     /* variant the adjoint uses now */
    int tuned;           /* 1 once the variants have been timed */
    size_t device_bytes; /* device memory held by the plan */
    int fold_lines;      /* folded forward: image lines staged per shared-memory strip */
    int fold_async;      /* folded forward: 1 if strips are double-buffered with cp.async */
    int fold2_group;     /* two-kernel folded forward: coefficients per CTA (0: unavailable) */
    int fold2_threads;   /* two-kernel folded forward: threads per CTA */
    int fold2_rays_per_thread; /* two-kernel folded forward: rays each thread marches */
    int fold2_lines;     /* two-kernel folded forward: strip lines */
    int fold2_split;     /* two-kernel folded forward: line chunks of the march */
    int fold2_async;     /* two-kernel folded forward: 1 if strips are double-buffered with cp.async */
    int fold_adj_angles; /* folded adjoint: distinct angles per pipeline stage */
    int fold2_angles;    /* two-kernel folded forward: distinct angles per CTA block */
    int fwd_variant_storage; /* forward variant of storage-typed calls (differs on BF16 plans) */
} dr_plan_info_t;

/* Describe the plan (host struct filled in). */
dr_status dr_plan_info(const dr_plan *plan, dr_plan_info_t *info);

/*
 * Wait for the plan's stream, then report any failure recorded by its
 * kernels (DR_ETIMEOUT if a bounded wait gave up) or by the CUDA runtime.
 * Clears the plan's device status word.
 */
dr_status dr_plan_sync(dr_plan *plan);

/*
 * Failure-path check of the library's bounded device-side waits (the paper
 * has no counterpart).  Launches, on the plan's stream, one CTA that waits
 * with the same bounded mbarrier wait the TMA pipelines use on a barrier
 * nothing arrives at; after limit_s seconds (0 < limit_s <= 2) the wait
 * gives up, records the failure in the plan's status word and the kernel
 * returns.  Then behaves as dr_plan_sync: DR_ETIMEOUT is the expected
 * result (the give-up path works and the context stays usable); DR_OK would
 * mean the wait did not give up.  DR_EINVAL for a NULL plan or a bad limit.
 */
dr_status dr_plan_wait_selftest(dr_plan *plan, double limit_s);

/*
 * Dynamic forward projection, Eq. (radapr) (Eq. Rfwd with Eq. repr):
 *     g[z][k][b] = sum_j phi_j(t_k) (R_{theta_k} u_j[z])(s_b)
 * u: device [nz][ny][nx][m], g: device [nz][K][ns] (overwritten).  u and g
 * must not overlap.  Asynchronous.
 */
dr_status dyn_radon_fwd(dr_plan *plan, const void *u, void *g);

/*
 * Adjoint (back-projection), Eq. (radadjapr) for a real basis:
 *     u_j[z] = beta * u_j[z] + sum_k phi_j(t_k) (R*_{theta_k} g[z][k])
 * R* is the exact transpose of dyn_radon_fwd's R.  g: device [nz][K][ns],
 * u: device [nz][ny][nx][m] (read when beta != 0, then overwritten).
 * Asynchronous.
 */
dr_status dyn_radon_adj(dr_plan *plan, const void *g, void *u, double beta);

/*
 * dyn_radon_adj for callers that may not allocate device memory at call
 * time -- code running while a stream is captured into a CUDA graph, or
 * applications whose memory policy forbids allocations after start-up.
 * The paper has no counterpart; it is a deployment variant.
 *     u_j[z] = beta * u_j[z] + sum_k phi_j(t_k) (R*_{theta_k} g[z][k])
 * computed by the half-turn fold, the same operator as dyn_radon_adj.
 * Instead of the plan's lazily allocated buffer, the folded data live in a
 * fixed 8 MiB (8388608-byte) device array inside the library, which every
 * GPU that loads the library holds until the process exits.  Requires an
 * F32 or BF16 plan with the fold available, the plan's device current, and
 * nz * U * ns * MS * 4 <= 8388608 bytes (U = distinct angles mod pi; MS =
 * 4 for m <= 4, 12 for m <= 12, 20 for m <= 16, 28 for m <= 24, 36 for
 * m <= 32): larger problems get DR_EINVAL with the size in dr_last_error();
 * call it per slab of slices instead.  Calls no cudaMalloc/cudaFree.
 * Set-up done by first calls: the first call on a device (and CUDA context)
 * looks up the array's device address (cudaGetSymbolAddress) and caches it
 * with the context's id; with lazy module loading (CUDA_MODULE_LOADING=LAZY,
 * the default) the array is reserved on that device by this first call, not
 * when the library loads; and the first call for each precision (F32, BF16)
 * and template size of m loads that kernel instantiation and raises its
 * dynamic shared-memory limit.  Make one call for every (precision, m) a
 * caller will use before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU (other streams or threads) race;
 * calls in order on one stream are safe.  Asynchronous.
 */
dr_status dyn_radon_adj_noalloc(dr_plan *plan, const void *g, void *u, double beta);

/*
 * Initial guess from filtered back-projection (Sec. 5 starts the iterations
 * from an FBP reconstruction with the Shepp-Logan filter).
 *   1. every projection row is filtered along s with the discrete Shepp-Logan
 *      kernel h(n) = -2 / (pi^2 (4 n^2 - 1)) (unit bin spacing, zero padded);
 *   2. projection k belongs to window w(k) = min(nw-1, max(0, floor(t_k nw)));
 *      the FBP image of window w is f_w = (pi / K_w) sum_{k in w} R*_k q_k
 *      (K_w projections spread over whole half-turns);
 *   3. u is the least-squares fit over the acquisition times:
 *      u = argmin sum_k || sum_j phi_j(t_k) u_j - f_{w(k)} ||^2,
 *      the minimum-norm one when the functions are dependent over the times
 *      (singular values of Phi below 1e-6 of the largest count as zero).
 * n_windows = 1 gives the static FBP of all projections spread over the
 * basis (the constant function's coefficients when it is in the span); one
 * window per half-turn gives the per-half-turn FBP frames of Sec. 5.
 * g: device [nz][K][ns] (storage precision), u: device [nz][ny][nx][m]
 * (overwritten).  The plan keeps scratch for the filtered data (nz K ns
 * compute-typed values, plus nx ny nz m floats for BF16 plans) until it is
 * destroyed.  Waits for the plan's stream before uploading its table, then
 * runs asynchronously.  DR_EINVAL if n_windows is outside [1, K] or every
 * basis function vanishes at every acquisition time.
 */
dr_status dr_fbp_init(dr_plan *plan, const void *g, void *u, int n_windows);

/*
 * 4D gradient of the synthesised frames, D = nabla_{lambda2} o PhiF
 * (Eq. TV1; frames f(t_l) = sum_j phi_j(t_l) u_j):  p = D u.
 * u: device [nz][ny][nx][m]; p: device [nz][nt][ny][nx][4] (overwritten).
 */
dr_status tv4d_grad(dr_plan *plan, const void *u, void *p, double lambda2);

/*
 * Adjoint of tv4d_grad (Sec. 3: K_2^* = -div_{lambda2}, then PhiF^T):
 *     u = beta * u + D^T p
 */
dr_status tv4d_grad_adj(dr_plan *plan, const void *p, void *u, double lambda2, double beta);

/*
 * The regulariser's normal operator, the D^T D term of the ADMM u-step
 * operator R*R + rho D^T D (D of Eq. TV1, D^T its adjoint, Sec. 3):
 *     out = beta * out + D^T D x
 * applied without forming D x: with G = PhiF^T PhiF and Lt = PhiF^T L_t PhiF
 * (m x m, built in double at plan time), D^T D = G (x) L_s + lambda2^2 Lt,
 * L_s / L_t the Neumann Laplacians in space and over the frames.
 * x, out: device [nz][ny][nx][m] in the plan's COMPUTE type (float for
 * DR_F32 and DR_BF16_F32ACC plans, double for DR_F64), distinct buffers.
 * DR_EINVAL for NULL pointers, x == out, or non-finite lambda2/beta.
 */
dr_status tv4d_normal(dr_plan *plan, const void *x, void *out, double lambda2, double beta);

/*
 * ADMM proximal and dual step on psi = D u (the shrink is the Moreau dual of
 * the projection that Sec. 3 uses as prox of sigma F_2^*):
 *     v = D u + mu/rho;  psi = v * max(0, 1 - (lambda1/rho)/|v|)  per (voxel, frame);
 *     mu <- mu + rho (D u - psi);  w <- psi - mu/rho.
 * u: device [nz][ny][nx][m]; mu (in/out), w (out): device [nz][nt][ny][nx][4].
 * primal_res: HOST double, nullable; when given the call synchronises and
 * stores ||D u - psi||_2 (accumulated in double).  rho > 0, lambda1 >= 0.
 */
dr_status tv4d_prox(dr_plan *plan, const void *u, void *mu, void *w, double rho, double lambda1,
                    double lambda2, double *primal_res);

typedef struct {
    dr_algo algo;
    int iters;              /* outer iterations, >= 0 */
    int n_cg;               /* ADMM: CG steps per u-step (warm started), >= 1 */
    double lambda1;         /* TV weight, >= 0 */
    double lambda2;         /* time-derivative weight inside the norm, >= 0 */
    double rho;             /* ADMM penalty; <= 0 selects 10 * lambda1 (or 1 if lambda1 = 0) */
    double cp_theta;        /* Chambolle-Pock extrapolation theta in [0, 1] */
    int power_iters;        /* Chambolle-Pock: power iterations for ||[R; D]||; <= 0 selects 100 */
    double *objective_out;  /* HOST [iters], nullable: Eq. (lr12) at u after each iteration */
    double *primal_res_out; /* HOST [iters], nullable: ADMM ||D u - psi|| after each iteration */
    double *op_norm_out;    /* HOST, nullable: Chambolle-Pock operator norm estimate used */
    double op_norm;         /* Chambolle-Pock: > 0 uses this ||[R; D]|| instead of the power iteration */
    void *state;            /* DEVICE, nullable: the solver's state besides u, in the plan's compute
                             * type (dr_plan_state_bytes), written at the end of the call, so that a
                             * later call can continue the iteration (checkpoint / resume) */
    int resume;             /* != 0: start from `state` instead of zero duals (needs state) */
} dr_solve_params;

/*
 * Bytes of the solver state admm_solve keeps besides u (dr_solve_params.state),
 * in the plan's compute type (float for DR_F32 / DR_BF16_F32ACC, double for
 * DR_F64), laid out as
 *   DR_ADMM_CG:         mu, w                 (two [nz][nt][ny][nx][4] fields)
 *   DR_CHAMBOLLE_POCK:  h2, h1, u~            ([nz][nt][ny][nx][4], [nz][K][ns],
 *                                              [nz][ny][nx][m])
 * A call with state != NULL writes its final state there; a call with
 * resume != 0 starts from it, so iters = a + b in one call and a then b with
 * the state carried over give the same iterates (Chambolle-Pock: pass the
 * same op_norm to both calls, e.g. the first call's op_norm_out).  u itself
 * is handed over in storage precision (bf16 for DR_BF16_F32ACC plans).  The
 * state is the caller's device memory; cp_solve_slabs takes none (DR_EINVAL).
 * Returns 0 for a NULL plan or an unknown algo.
 */
size_t dr_plan_state_bytes(const dr_plan *plan, dr_algo algo);

/* Fill params with defaults: ADMM-CG, 20 iterations, 4 CG steps, lambda1 = lambda2 = 1e-3... */
void dr_solve_params_default(dr_solve_params *params);

/*
 * Solve Eq. (lr12) for the coefficients u.
 *   DR_ADMM_CG: split psi = D u; per iteration n_cg CG steps on
 *       (R*R + rho D^T D) u = R* g + rho D^T (psi - mu/rho)   (warm start,
 *       explicit residual, early stop when <r,r> = 0 or <p,Ap> <= 0), then
 *       the tv4d_prox step.  mu = psi = 0 at the start (or the state of an
 *       earlier call: dr_solve_params.state / resume).
 *   DR_CHAMBOLLE_POCK: Sec. 3, Fig. 2 with h1 = h2 = 0 (or a resumed state) at the start and
 *       tau = sigma = 0.99 / L, L = ||[R; D]|| from power_iters power
 *       iterations started from a SplitMix64 vector (seed 1809).
 * g: [nz][K][ns]; u: [nz][ny][nx][m], initial guess in, result out.  Either
 * may be a host or a device pointer (host buffers are copied inside the
 * call).  The call synchronises the plan's stream before returning; inner
 * products, step sizes and residuals are kept on the device in double, and
 * each iteration is replayed as one CUDA graph.  Allocates the workspace on
 * first use (kept by the plan).  Returns DR_ETIMEOUT if a device wait gave up.
 */
dr_status admm_solve(dr_plan *plan, const void *g, void *u, const dr_solve_params *params);

/*
 * Several independent reconstructions at once (uneven sizes, bases,
 * precisions and iteration counts allowed).  Job j solves Eq. (lr12) for
 * plans[j], g[j], u[j], params[j] exactly as admm_solve would; the first
 * iteration of every job runs eagerly, then each iteration of all jobs still
 * running is replayed as ONE CUDA graph with one branch per job (forked from
 * a root stream and joined back), so the jobs' kernels overlap on the
 * device.  Each job keeps its own plan workspace, scalars and reduction
 * order, so its result is bit-for-bit that of a separate admm_solve call.
 * Plans must be distinct and on the same device; arrays have njobs entries.
 * Synchronises before returning.
 */
dr_status admm_solve_batch(int njobs, dr_plan *const *plans, const void *const *g, void *const *u,
                           const dr_solve_params *params);

/*
 * Chambolle-Pock (Sec. 3, Fig. 2) for a volume kept in HOST memory and
 * streamed through the GPU in slabs of slab_nz slices, the scheme of Sec. 6:
 * each slab is copied in with the slice above it (for the forward z
 * difference of D), steps 3-6 run on it, and it is copied out, with the
 * copies of the neighbouring slabs overlapping the computation on separate
 * streams.  The updated dual on the slice below a slab is carried over on the
 * device from the previous slab.  With the same operator norm (params->op_norm
 * > 0) the result is bit-identical to admm_solve with DR_CHAMBOLLE_POCK and
 * the same projector variants; otherwise the norm comes from a streamed power
 * iteration (params->power_iters passes over the volume), equal to the
 * in-core estimate up to rounding.
 *   plan     the whole volume's plan (nz = all slices); its stream is
 *            synchronised first and the plan must not be used concurrently
 *   g        HOST [nz][K][ns] storage precision (copied to pinned memory once
 *            if it is pageable)
 *   u        HOST [nz][ny][nx][m] storage precision: initial guess in, result out
 *   params   algo must be DR_CHAMBOLLE_POCK (ADMM-CG needs whole-volume inner
 *            products inside every CG step); objective_out / op_norm_out as
 *            for admm_solve
 *   slab_nz  slices per slab (>= 1; device memory grows with it)
 * Host memory: pinned copies of u, u~, h1 and h2 (compute precision) for the
 * whole volume.  Device memory: cp_solve_slabs_device_bytes().  Synchronous.
 * DR_EINVAL for device pointers or bad parameters, DR_ENOMEM if the slab
 * buffers do not fit, DR_ENOTCONV for non-finite results.
 */
dr_status cp_solve_slabs(dr_plan *plan, const void *g, void *u, const dr_solve_params *params, int slab_nz);

/* Device bytes cp_solve_slabs allocates for this plan, slab thickness and
 * parameters (0 on bad arguments). */
size_t cp_solve_slabs_device_bytes(dr_plan *plan, int slab_nz, const dr_solve_params *params);

/* ------------------------------------------------------------------------ */
/* Serving: a request loop with device-memory-budget admission.             */
/* ------------------------------------------------------------------------ */
typedef struct dr_server dr_server;

enum { DR_JOB_QUEUED = 0, DR_JOB_RUNNING = 1, DR_JOB_DONE = 2, DR_JOB_FAILED = 3, DR_JOB_CANCELED = 4 };

/* One reconstruction request.  theta and t are copied at submission; g, u
 * and the output pointers inside params (host or device memory) are the
 * caller's and must stay valid until the job has finished. */
typedef struct {
    int nx, ny, nz, ns, K;
    const double *theta;    /* [K] radians */
    const double *t;        /* [K] in [0, 1) */
    dr_basis basis;
    int m, nt;
    dr_precision prec;
    dr_solve_params params;
    const void *g;          /* [nz][K][ns] data */
    void *u;                /* [nz][ny][nx][m] initial guess in, result out */
} dr_job_desc;

typedef struct {
    int state;              /* DR_JOB_* */
    dr_status status;
    double latency_s;       /* completion - submission */
    double queue_s;         /* start - submission */
    size_t device_bytes;    /* memory the job was admitted with */
    int slab_nz;            /* 0: whole volume on the device; > 0: streamed through
                             * the GPU in slabs of this many slices (cp_solve_slabs) */
} dr_job_result;

typedef struct {
    int64_t completed, failed, canceled, queued;
    int active;
    double p50_latency_s, p99_latency_s;
    size_t peak_device_bytes, budget_bytes;
    double voxel_projection_per_s;  /* projector work of completed jobs / busy span */
} dr_server_stats_t;

/* Device bytes a job is admitted with (host arithmetic only, no CUDA call):
 * plan tables, reduction slots, folded-data scratch, solver workspace and
 * the staging copies of host inputs. */
size_t dr_job_device_bytes(const dr_job_desc *desc);

/* Device bytes of the same job streamed in slabs of slab_nz slices
 * (cp_solve_slabs; host arithmetic only, an upper bound). */
size_t dr_job_slab_device_bytes(const dr_job_desc *desc, int slab_nz);

/* Start a server on `device` with `slots` worker threads (jobs that may run
 * at once) and a device-memory budget in bytes for all running jobs. */
dr_status dr_server_create(dr_server **out, int device, size_t budget_bytes, int slots);

/* Queue a job; returns its id.  A Chambolle-Pock job on host buffers whose
 * whole-volume state does not fit the budget is streamed through the GPU in
 * the thickest slabs that fit (Sec. 6); DR_ENOMEM if even one-slice slabs (or,
 * for other jobs, the whole volume) cannot fit the budget alone.  Queued jobs
 * are admitted in order, a later job that fits may pass a head job that does
 * not (backfill); admitted jobs keep their state on the device (or stream it)
 * and run concurrently, each with its own plan and stream. */
dr_status dr_server_submit(dr_server *server, const dr_job_desc *desc, int64_t *job_id);

/* Cancel a job.  A queued job is removed at once; a running ADMM-CG or
 * in-core Chambolle-Pock job stops between iterations (within about two
 * iterations: a serving job's solve keeps at most two iterations in flight)
 * and ends with state DR_JOB_CANCELED and status DR_ECANCELED, u holding no
 * defined result; a slab-streamed job runs to the end.  DR_EINVAL for an
 * unknown or finished job. */
dr_status dr_server_cancel(dr_server *server, int64_t job_id);

/* Wait up to timeout_s seconds (< 0: no limit) for a job; fills res
 * (nullable) and returns the job's status (DR_ETIMEOUT if still running). */
dr_status dr_server_wait(dr_server *server, int64_t job_id, double timeout_s, dr_job_result *res);

/* Counters and latency percentiles of completed jobs. */
dr_status dr_server_stats(dr_server *server, dr_server_stats_t *stats);

/* Finish all queued and running jobs, stop the workers, free the server. */
dr_status dr_server_destroy(dr_server *server);

/* Message of the last failed call on this thread ("" if none). */
const char *dr_last_error(void);

/* Library version string. */
const char *dr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DYNRECON_H */
