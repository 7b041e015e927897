/*
 * dynrecon_oracle.c -- plain FP64 CPU oracle for the dynamic (4D) tomography
 * hot path of Nikitin, Carlsson, Andersson, Mokso, "Four-dimensional
 * tomographic reconstruction by time domain decomposition" (arXiv 1809.09725).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * Everything is double precision, written as the plain definition, with no
 * blocking, fusion or reordering beyond what the definition states.  Compile
 * with -ffp-contract=off so that no multiply-add is fused.
 *
 * Geometry (the paper fixes only the continuous line x cos(theta) + y sin(theta)
 * = s of Eq. (Rfwd), Sec. 2; the discretisation below is this project's reading):
 *   pixel centres  x_i = i - (nx-1)/2,  y_j = j - (ny-1)/2   (unit pixels)
 *   detector bins  s_b = b - (ns-1)/2                        (unit spacing)
 *   slices z are independent (parallel beam).
 *
 * Array layouts (row-major, last index fastest):
 *   u  [nz][ny][nx][m]     temporal-basis coefficient volumes u_j (Eq. repr)
 *   g  [nz][K][ns]         projection data g(theta_k, s_b, z)
 *   F  [nz][ny][nx][nt]    frames f(x, t_l)
 *   p  [nz][ny][nx][nt][4] 4-vector fields (d/dx, d/dy, d/dz, lambda2 d/dt)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

/* ------------------------------------------------------------------------- */
/* Temporal bases (Sec. 4, Eq. repr; Sec. 5 uses a Fourier basis; Sec. 4     */
/* and Sec. 8 name Haar wavelets and Heaviside step functions).              */
/* kind 0: real Fourier  phi_0 = 1, phi_{2i-1} = cos(2 pi i t),              */
/*                       phi_{2i} = sin(2 pi i t)                            */
/* kind 1: shifted Legendre  phi_j(t) = P_j(2t - 1), three-term recurrence   */
/*         (n+1) P_{n+1}(x) = (2n+1) x P_n(x) - n P_{n-1}(x).                */
/* kind 2: Haar  phi_0 = 1; for j >= 1 write j = 2^lev + pos (0 <= pos <    */
/*         2^lev): phi_j(t) = +1 on [pos, pos + 1/2) / 2^lev, -1 on          */
/*         [pos + 1/2, pos + 1) / 2^lev, 0 elsewhere (unnormalised).          */
/* kind 3: Heaviside  phi_0 = 1, phi_j(t) = 1 if t >= j/m else 0.            */
/* kind 4: complex Fourier of Sec. 5, phi_j(t) = exp(2 pi i t (j - M/2)),    */
/*         j = 0..M-1, carried as m = 2M real channels: the object           */
/*         f(t) = Re sum_j u_j phi_j(t) with u_j = a_j + i b_j is            */
/*         sum_j a_j cos(w_j t) - b_j sin(w_j t), w_j = 2 pi (j - M/2), so   */
/*         channel 2j = cos(w_j t), channel 2j+1 = -sin(w_j t).              */
/* out[n][m] = phi_j(t[i]).                                                  */
/* ------------------------------------------------------------------------- */
static double haar(int j, double t)
{
    if (j == 0) return 1.0;
    int lev = 0;
    while ((2 << lev) <= j) ++lev;
    int pos = j - (1 << lev);
    double x = t * (double)(1 << lev) - (double)pos; /* position inside the support */
    if (x >= 0.0 && x < 0.5) return 1.0;
    if (x >= 0.5 && x < 1.0) return -1.0;
    return 0.0;
}

int or_basis_table(int kind, int m, const double *t, i64 n, double *out)
{
    if (m < 1 || kind < 0 || kind > 4 || (kind == 4 && m % 2 != 0)) return -1;
    for (i64 i = 0; i < n; ++i) {
        double *row = out + i * m;
        if (kind == 4) {
            int M = m / 2;
            for (int j = 0; j < M; ++j) {
                double w = 2.0 * M_PI * (double)(j - M / 2);
                row[2 * j] = cos(w * t[i]);
                row[2 * j + 1] = -sin(w * t[i]);
            }
        } else if (kind == 2) {
            for (int j = 0; j < m; ++j) row[j] = haar(j, t[i]);
        } else if (kind == 3) {
            for (int j = 0; j < m; ++j) row[j] = (j == 0 || t[i] >= (double)j / (double)m) ? 1.0 : 0.0;
        } else if (kind == 0) {
            row[0] = 1.0;
            for (int j = 1; j < m; ++j) {
                int freq = (j + 1) / 2;
                double arg = 2.0 * M_PI * (double)freq * t[i];
                row[j] = (j % 2 == 1) ? cos(arg) : sin(arg);
            }
        } else {
            double x = 2.0 * t[i] - 1.0;
            row[0] = 1.0;
            if (m > 1) row[1] = x;
            for (int j = 1; j + 1 < m; ++j)
                row[j + 1] = ((2.0 * j + 1.0) * x * row[j] - (double)j * row[j - 1]) / (double)(j + 1);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gram-Schmidt orthonormalisation of a basis over the acquisition times     */
/* (Sec. 4 suggests it to make a basis orthonormal): modified Gram-Schmidt   */
/* on the columns of Phi[K][m] (samples phi_j(t_k)) gives Phi = Q Rm with Q  */
/* orthonormal over the samples; the new basis is phi~ = phi Rm^{-1},        */
/* applied to Phi (becomes Q) and to any other table of the same functions   */
/* (PhiF[nt][m]).  Returns -1 if a column is dependent on the previous ones. */
/* ------------------------------------------------------------------------- */
int or_orthonormalise(double *Phi, i64 K, int m, double *PhiF, i64 nt)
{
    double *Rm = (double *)calloc((size_t)m * m, sizeof(double));
    for (int j = 0; j < m; ++j) {
        for (int i = 0; i < j; ++i) {
            double d = 0.0;
            for (i64 k = 0; k < K; ++k) d += Phi[k * m + i] * Phi[k * m + j];
            Rm[i * m + j] = d;
            for (i64 k = 0; k < K; ++k) Phi[k * m + j] -= d * Phi[k * m + i];
        }
        double nrm = 0.0;
        for (i64 k = 0; k < K; ++k) nrm += Phi[k * m + j] * Phi[k * m + j];
        nrm = sqrt(nrm);
        if (!(nrm > 1e-12)) {
            free(Rm);
            return -1;
        }
        Rm[j * m + j] = nrm;
        for (i64 k = 0; k < K; ++k) Phi[k * m + j] /= nrm;
    }
    /* PhiF <- PhiF Rm^{-1}: solve X Rm = PhiF row by row (Rm upper triangular) */
    for (i64 l = 0; l < nt; ++l) {
        double *row = PhiF + l * m;
        for (int j = 0; j < m; ++j) {
            double v = row[j];
            for (int i = 0; i < j; ++i) v -= row[i] * Rm[i * m + j];
            row[j] = v / Rm[j * m + j];
        }
    }
    free(Rm);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Joseph ray-driven projection of one 2D image F[ny][nx] at angle theta.    */
/* Discrete counterpart of the static Radon transform R used in Eq. (radapr) */
/* If |cos| >= |sin|: one sample per row j, at x* = (s - y_j sin)/cos,       */
/* linear interpolation between the two pixels of that row that bracket x*   */
/* (pixels outside the grid are zero), sum times 1/|cos|.                    */
/* Otherwise the same with the roles of x and y exchanged, times 1/|sin|.    */
/* ------------------------------------------------------------------------- */
static double pix(const double *F, int nx, int ny, i64 i, i64 j)
{
    if (i < 0 || i >= nx || j < 0 || j >= ny) return 0.0;
    return F[j * nx + i];
}

void or_joseph_fwd_slice(const double *F, int nx, int ny, double theta, int ns, double *out)
{
    double c = cos(theta), s = sin(theta);
    for (int b = 0; b < ns; ++b) {
        double sb = (double)b - 0.5 * (ns - 1);
        double acc = 0.0;
        if (fabs(c) >= fabs(s)) {
            for (int j = 0; j < ny; ++j) {
                double yj = (double)j - 0.5 * (ny - 1);
                double xi = (sb - yj * s) / c + 0.5 * (nx - 1);
                double i0 = floor(xi);
                double w = xi - i0;
                acc += (1.0 - w) * pix(F, nx, ny, (i64)i0, j) + w * pix(F, nx, ny, (i64)i0 + 1, j);
            }
            out[b] = acc / fabs(c);
        } else {
            for (int i = 0; i < nx; ++i) {
                double xi_ = (double)i - 0.5 * (nx - 1);
                double eta = (sb - xi_ * c) / s + 0.5 * (ny - 1);
                double j0 = floor(eta);
                double w = eta - j0;
                acc += (1.0 - w) * pix(F, nx, ny, i, (i64)j0) + w * pix(F, nx, ny, i, (i64)j0 + 1);
            }
            out[b] = acc / fabs(s);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Exact transpose of or_joseph_fwd_slice, written pixel-driven (gather).    */
/* A Joseph sample at distance d (in the stepping axis) from a pixel centre  */
/* gives that pixel the weight max(0, 1 - d); in the |cos|>=|sin| case the   */
/* sample of bin b in row j lies at x* with x* - x_i = (s_b - p)/cos, where  */
/* p = x_i cos + y_j sin, and symmetrically for the other case.  With        */
/* c = max(|cos|, |sin|) the pixel therefore receives                        */
/*     sum_b g[b] * max(0, 1 - |s_b - p| / c) / c.                           */
/* Only bins with |s_b - p| < c can contribute; the loop visits that range.  */
/* ------------------------------------------------------------------------- */
void or_joseph_adj_slice(const double *g, int ns, double theta, int nx, int ny, double *out)
{
    double c = cos(theta), s = sin(theta);
    double cm = fabs(c) >= fabs(s) ? fabs(c) : fabs(s);
    for (int j = 0; j < ny; ++j) {
        double yj = (double)j - 0.5 * (ny - 1);
        for (int i = 0; i < nx; ++i) {
            double xi = (double)i - 0.5 * (nx - 1);
            double p = xi * c + yj * s;
            double pos = p + 0.5 * (ns - 1); /* p in bin-index units */
            i64 blo = (i64)ceil(pos - cm) - 1;
            i64 bhi = (i64)floor(pos + cm) + 1;
            if (blo < 0) blo = 0;
            if (bhi > ns - 1) bhi = ns - 1;
            double acc = 0.0;
            for (i64 b = blo; b <= bhi; ++b) {
                double sb = (double)b - 0.5 * (ns - 1);
                double wt = 1.0 - fabs(sb - p) / cm;
                if (wt > 0.0) acc += g[b] * wt / cm;
            }
            out[j * nx + i] = acc;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Dynamic projection, Eq. (Rfwd) with the decomposition of Eq. (repr):      */
/* at each acquisition k the object state f(., t_k) = sum_j phi_j(t_k) u_j   */
/* is formed and projected at theta_k.  By linearity this equals Eq. (radapr)*/
/*   g[z][k] = sum_j phi_j(t_k) R_{theta_k} u_j[z].                          */
/* Phi[K][m] = phi_j(t_k).                                                   */
/* ------------------------------------------------------------------------- */
void or_dyn_fwd(const double *u, int nx, int ny, int nz, int m, int K,
                const double *theta, const double *Phi, int ns, double *g)
{
    i64 npix = (i64)nx * ny;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int z = 0; z < nz; ++z) {
        for (int k = 0; k < K; ++k) {
            double *frame = (double *)malloc(sizeof(double) * npix);
            for (i64 q = 0; q < npix; ++q) {
                double v = 0.0;
                for (int j = 0; j < m; ++j)
                    v += Phi[(i64)k * m + j] * u[((i64)z * npix + q) * m + j];
                frame[q] = v;
            }
            or_joseph_fwd_slice(frame, nx, ny, theta[k], ns, g + ((i64)z * K + k) * ns);
            free(frame);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Adjoint, Eq. (radadjapr) for a real basis (hat phi_j = phi_j):            */
/*   u_j[z] = sum_k phi_j(t_k) R*_{theta_k} g[z][k]                          */
/* with R* the exact transpose above.                                        */
/* ------------------------------------------------------------------------- */
void or_dyn_adj(const double *g, int nx, int ny, int nz, int m, int K,
                const double *theta, const double *Phi, int ns, double *u)
{
    i64 npix = (i64)nx * ny;
    memset(u, 0, sizeof(double) * (size_t)(nz * npix * m));
    /* pixel-driven: every pixel sums its projections in ascending k */
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int z = 0; z < nz; ++z) {
        for (int j = 0; j < ny; ++j) {
            double yj = (double)j - 0.5 * (ny - 1);
            for (int k = 0; k < K; ++k) {
                const double *gk = g + ((i64)z * K + k) * ns;
                double c = cos(theta[k]), s = sin(theta[k]);
                double cm = fabs(c) >= fabs(s) ? fabs(c) : fabs(s);
                for (int i = 0; i < nx; ++i) {
                    double xi = (double)i - 0.5 * (nx - 1);
                    double p = xi * c + yj * s;
                    double pos = p + 0.5 * (ns - 1);
                    i64 blo = (i64)ceil(pos - cm) - 1;
                    i64 bhi = (i64)floor(pos + cm) + 1;
                    if (blo < 0) blo = 0;
                    if (bhi > ns - 1) bhi = ns - 1;
                    double acc = 0.0;
                    for (i64 b = blo; b <= bhi; ++b) {
                        double sb = (double)b - 0.5 * (ns - 1);
                        double wt = 1.0 - fabs(sb - p) / cm;
                        if (wt > 0.0) acc += gk[b] * wt / cm;
                    }
                    double *uq = u + ((i64)z * npix + (i64)j * nx + i) * m;
                    for (int jj = 0; jj < m; ++jj) uq[jj] += Phi[(i64)k * m + jj] * acc;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Frames on the reconstruction time grid t_l = l / nt, l = 0..nt-1 (one     */
/* frame per half-turn by default, Sec. 4 Eq. discrt):                       */
/*   F[.][l] = sum_j PhiF[l][j] u_j       and its transpose.                 */
/* ------------------------------------------------------------------------- */
void or_frames(const double *u, i64 nvox, int m, const double *PhiF, int nt, double *F)
{
    for (i64 v = 0; v < nvox; ++v)
        for (int l = 0; l < nt; ++l) {
            double a = 0.0;
            for (int j = 0; j < m; ++j) a += PhiF[(i64)l * m + j] * u[v * m + j];
            F[v * nt + l] = a;
        }
}

void or_frames_T(const double *F, i64 nvox, int m, const double *PhiF, int nt, double *u)
{
    for (i64 v = 0; v < nvox; ++v)
        for (int j = 0; j < m; ++j) {
            double a = 0.0;
            for (int l = 0; l < nt; ++l) a += PhiF[(i64)l * m + j] * F[v * nt + l];
            u[v * m + j] = a;
        }
}

/* ------------------------------------------------------------------------- */
/* Gradient nabla_{lambda2} of Eq. (TV1) with forward differences and unit   */
/* spacing (Sec. 4 for the time difference); the difference across the last  */
/* index of each dimension is zero (Neumann).                                */
/* ------------------------------------------------------------------------- */
#define FIDX(z, y, x, l) ((((i64)(z) * ny + (y)) * nx + (x)) * nt + (l))

void or_grad4(const double *F, int nx, int ny, int nz, int nt, double lambda2, double *p)
{
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int l = 0; l < nt; ++l) {
                    double f = F[FIDX(z, y, x, l)];
                    double *q = p + FIDX(z, y, x, l) * 4;
                    q[0] = (x + 1 < nx) ? F[FIDX(z, y, x + 1, l)] - f : 0.0;
                    q[1] = (y + 1 < ny) ? F[FIDX(z, y + 1, x, l)] - f : 0.0;
                    q[2] = (z + 1 < nz) ? F[FIDX(z + 1, y, x, l)] - f : 0.0;
                    q[3] = (l + 1 < nt) ? lambda2 * (F[FIDX(z, y, x, l + 1)] - f) : 0.0;
                }
}

/* div_{lambda2} = -(nabla_{lambda2})^T (Sec. 3, K_2^* = -div): backward     */
/* differences with the boundary rule matching or_grad4.                     */
void or_div4(const double *p, int nx, int ny, int nz, int nt, double lambda2, double *F)
{
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int l = 0; l < nt; ++l) {
                    const double *q = p + FIDX(z, y, x, l) * 4;
                    double d = 0.0;
                    if (x + 1 < nx) d += q[0];
                    if (x > 0) d -= p[FIDX(z, y, x - 1, l) * 4 + 0];
                    if (y + 1 < ny) d += q[1];
                    if (y > 0) d -= p[FIDX(z, y - 1, x, l) * 4 + 1];
                    if (z + 1 < nz) d += q[2];
                    if (z > 0) d -= p[FIDX(z - 1, y, x, l) * 4 + 2];
                    if (l + 1 < nt) d += lambda2 * q[3];
                    if (l > 0) d -= lambda2 * p[FIDX(z, y, x, l - 1) * 4 + 3];
                    F[FIDX(z, y, x, l)] = d;
                }
}
#undef FIDX

/* D = nabla_{lambda2} o PhiF  (coefficients -> 4-vector field on frames).   */
void or_D(const double *u, int nx, int ny, int nz, int m, const double *PhiF, int nt,
          double lambda2, double *p)
{
    i64 nvox = (i64)nx * ny * nz;
    double *F = (double *)malloc(sizeof(double) * nvox * nt);
    or_frames(u, nvox, m, PhiF, nt, F);
    or_grad4(F, nx, ny, nz, nt, lambda2, p);
    free(F);
}

/* D^T = PhiF^T o (-div_{lambda2}). */
void or_DT(const double *p, int nx, int ny, int nz, int m, const double *PhiF, int nt,
           double lambda2, double *u)
{
    i64 nvox = (i64)nx * ny * nz;
    double *F = (double *)malloc(sizeof(double) * nvox * nt);
    or_div4(p, nx, ny, nz, nt, lambda2, F);
    for (i64 q = 0; q < nvox * nt; ++q) F[q] = -F[q];
    or_frames_T(F, nvox, m, PhiF, nt, u);
    free(F);
}

/* ------------------------------------------------------------------------- */
/* Pointwise proximal maps on 4-vectors.                                     */
/* shrink: argmin_psi kappa |psi| + 1/2 |v - psi|^2 = v max(0, 1 - kappa/|v|)*/
/* project: onto the ball |h| <= lam, the prox of the conjugate of           */
/*          lam |.| (Sec. 3, prox of sigma F_2^*), read pointwise.           */
/* ------------------------------------------------------------------------- */
void or_shrink4(const double *v, double kappa, double *out)
{
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
    double f = 0.0;
    if (n > 0.0) {
        f = 1.0 - kappa / n;
        if (f < 0.0) f = 0.0;
    }
    for (int c = 0; c < 4; ++c) out[c] = v[c] * f;
}

void or_project4(const double *h, double lam, double *out)
{
    /* h / max(1, |h|/lam), written so that lam = 0 gives the point 0 */
    double n = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2] + h[3] * h[3]);
    for (int c = 0; c < 4; ++c) out[c] = (n <= lam) ? h[c] : h[c] * (lam / n);
}

/* ------------------------------------------------------------------------- */
/* ADMM proximal/dual step on psi = D u:                                     */
/*   v = D u + mu/rho;  psi = shrink(v, lambda1/rho);  mu += rho (D u - psi);*/
/*   w = psi - mu/rho.                                                       */
/* Returns sum |D u| (for the objective) and ||D u - psi||^2.                */
/* ------------------------------------------------------------------------- */
void or_tv4d_prox(const double *u, double *mu, double *w, int nx, int ny, int nz, int m,
                  const double *PhiF, int nt, double rho, double lambda1, double lambda2,
                  double *tv_sum, double *primal_sq)
{
    i64 n = (i64)nx * ny * nz * nt;
    double *Du = (double *)malloc(sizeof(double) * n * 4);
    or_D(u, nx, ny, nz, m, PhiF, nt, lambda2, Du);
    double tv = 0.0, pr = 0.0;
    for (i64 q = 0; q < n; ++q) {
        double v[4], psi[4];
        double *d = Du + q * 4;
        tv += sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3]);
        for (int c = 0; c < 4; ++c) v[c] = d[c] + mu[q * 4 + c] / rho;
        or_shrink4(v, lambda1 / rho, psi);
        for (int c = 0; c < 4; ++c) {
            double r = d[c] - psi[c];
            pr += r * r;
            mu[q * 4 + c] += rho * r;
            w[q * 4 + c] = psi[c] - mu[q * 4 + c] / rho;
        }
    }
    free(Du);
    if (tv_sum) *tv_sum = tv;
    if (primal_sq) *primal_sq = pr;
}

/* ------------------------------------------------------------------------- */
/* Problem description shared by the solvers.                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz, ns, K, m, nt;
    const double *theta; /* [K] */
    const double *Phi;   /* [K][m]  phi_j(t_k)   */
    const double *PhiF;  /* [nt][m] phi_j(l/nt)  */
} or_problem;

static i64 nu_of(const or_problem *P) { return (i64)P->nx * P->ny * P->nz * P->m; }
static i64 ng_of(const or_problem *P) { return (i64)P->nz * P->K * P->ns; }
static i64 np_of(const or_problem *P) { return (i64)P->nx * P->ny * P->nz * P->nt * 4; }

static double dot(const double *a, const double *b, i64 n)
{
    double s = 0.0;
    for (i64 i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Objective of Eq. (lr12) in the coefficient variables:                    */
/*   1/2 ||R u - g||^2 + lambda1 sum_{x,l} |D u|(x,l).                       */
double or_objective(const or_problem *P, const double *g, const double *u, double lambda1,
                    double lambda2)
{
    i64 ng = ng_of(P), np = np_of(P);
    double *Ru = (double *)malloc(sizeof(double) * ng);
    double *Du = (double *)malloc(sizeof(double) * np);
    or_dyn_fwd(u, P->nx, P->ny, P->nz, P->m, P->K, P->theta, P->Phi, P->ns, Ru);
    double fid = 0.0;
    for (i64 i = 0; i < ng; ++i) fid += (Ru[i] - g[i]) * (Ru[i] - g[i]);
    or_D(u, P->nx, P->ny, P->nz, P->m, P->PhiF, P->nt, lambda2, Du);
    double tv = 0.0;
    for (i64 q = 0; q < np / 4; ++q) {
        double *d = Du + q * 4;
        tv += sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + d[3] * d[3]);
    }
    free(Ru);
    free(Du);
    return 0.5 * fid + lambda1 * tv;
}

/* A x = R* R x + rho D^T D x  (the ADMM u-step normal operator). */
static void apply_A(const or_problem *P, const double *x, double rho, double lambda2,
                    double *out, double *tg, double *tp, double *tu)
{
    i64 nu = nu_of(P);
    or_dyn_fwd(x, P->nx, P->ny, P->nz, P->m, P->K, P->theta, P->Phi, P->ns, tg);
    or_dyn_adj(tg, P->nx, P->ny, P->nz, P->m, P->K, P->theta, P->Phi, P->ns, out);
    or_D(x, P->nx, P->ny, P->nz, P->m, P->PhiF, P->nt, lambda2, tp);
    or_DT(tp, P->nx, P->ny, P->nz, P->m, P->PhiF, P->nt, lambda2, tu);
    for (i64 i = 0; i < nu; ++i) out[i] += rho * tu[i];
}

/* ------------------------------------------------------------------------- */
/* ADMM with a conjugate-gradient u-step (the solver the workload names; the */
/* paper solves the same model, Eq. (lr12), with Chambolle-Pock).            */
/* Split psi = D u.  Per outer iteration:                                    */
/*   u   <- n_cg steps of linear CG (Hestenes-Stiefel) on                    */
/*          (R*R + rho D^T D) u = R* g + rho D^T (psi - mu/rho), warm start, */
/*          residual formed explicitly at the start, stopped early when      */
/*          <r,r> = 0 or <p,Ap> <= 0;                                        */
/*   psi <- shrink(D u + mu/rho, lambda1/rho);  mu <- mu + rho (D u - psi).  */
/* u is the initial guess on entry and the result on exit; mu = psi = 0 at   */
/* the start.  objective[n] is Eq. (lr12) at u after iteration n.            */
/* ------------------------------------------------------------------------- */
int or_admm_cg(const or_problem *P, const double *g, double *u, int iters, int n_cg,
               double lambda1, double lambda2, double rho, double *objective,
               double *primal_res)
{
    i64 nu = nu_of(P), ng = ng_of(P), np = np_of(P);
    double *mu = (double *)calloc((size_t)np, sizeof(double));
    double *w = (double *)calloc((size_t)np, sizeof(double));
    double *b = (double *)malloc(sizeof(double) * nu);
    double *r = (double *)malloc(sizeof(double) * nu);
    double *pv = (double *)malloc(sizeof(double) * nu);
    double *q = (double *)malloc(sizeof(double) * nu);
    double *tu = (double *)malloc(sizeof(double) * nu);
    double *tg = (double *)malloc(sizeof(double) * ng);
    double *tp = (double *)malloc(sizeof(double) * np);
    if (!mu || !w || !b || !r || !pv || !q || !tu || !tg || !tp) return -2;

    for (int it = 0; it < iters; ++it) {
        /* b = R* g + rho D^T w,  w = psi - mu/rho */
        or_dyn_adj(g, P->nx, P->ny, P->nz, P->m, P->K, P->theta, P->Phi, P->ns, b);
        or_DT(w, P->nx, P->ny, P->nz, P->m, P->PhiF, P->nt, lambda2, tu);
        for (i64 i = 0; i < nu; ++i) b[i] += rho * tu[i];
        /* r = b - A u */
        apply_A(P, u, rho, lambda2, q, tg, tp, tu);
        for (i64 i = 0; i < nu; ++i) r[i] = b[i] - q[i];
        memcpy(pv, r, sizeof(double) * nu);
        double rr = dot(r, r, nu);
        for (int c = 0; c < n_cg; ++c) {
            if (rr == 0.0) break;
            apply_A(P, pv, rho, lambda2, q, tg, tp, tu);
            double pq = dot(pv, q, nu);
            if (!(pq > 0.0)) break;
            double alpha = rr / pq;
            for (i64 i = 0; i < nu; ++i) u[i] += alpha * pv[i];
            for (i64 i = 0; i < nu; ++i) r[i] -= alpha * q[i];
            double rr_new = dot(r, r, nu);
            double beta = rr_new / rr;
            for (i64 i = 0; i < nu; ++i) pv[i] = r[i] + beta * pv[i];
            rr = rr_new;
        }
        double pr2 = 0.0;
        or_tv4d_prox(u, mu, w, P->nx, P->ny, P->nz, P->m, P->PhiF, P->nt, rho, lambda1, lambda2,
                     NULL, &pr2);
        if (primal_res) primal_res[it] = sqrt(pr2);
        if (objective) objective[it] = or_objective(P, g, u, lambda1, lambda2);
    }
    free(mu); free(w); free(b); free(r); free(pv); free(q); free(tu); free(tg); free(tp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Counter-based SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the i-th      */
/* output of the generator seeded with `seed` is mix(seed + (i+1) * gamma).  */
/* Returns a double uniform in [0, 1) from the top 53 bits.                  */
/* ------------------------------------------------------------------------- */
double or_splitmix_uniform(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------------------------------------- */
/* Operator norm L = ||[R; D]|| by power iteration on R*R + D^T D.  The      */
/* start vector is x_i = 0.5 + U_i, U_i the SplitMix64 stream with seed      */
/* 1809; a symmetric start (all ones) can be orthogonal to the top singular  */
/* vector, e.g. when D couples slices with opposite signs.                   */
/* ------------------------------------------------------------------------- */
double or_power_norm(const or_problem *P, double lambda2, int iters)
{
    i64 nu = nu_of(P), ng = ng_of(P), np = np_of(P);
    double *x = (double *)malloc(sizeof(double) * nu);
    double *y = (double *)malloc(sizeof(double) * nu);
    double *tu = (double *)malloc(sizeof(double) * nu);
    double *tg = (double *)malloc(sizeof(double) * ng);
    double *tp = (double *)malloc(sizeof(double) * np);
    for (i64 i = 0; i < nu; ++i) x[i] = 0.5 + or_splitmix_uniform(1809u, (uint64_t)i);
    double x2 = sqrt(dot(x, x, nu));
    for (i64 i = 0; i < nu; ++i) x[i] /= x2;
    double lam = 0.0;
    for (int it = 0; it < iters; ++it) {
        apply_A(P, x, 1.0, lambda2, y, tg, tp, tu);
        lam = sqrt(dot(y, y, nu));
        if (lam == 0.0) break;
        for (i64 i = 0; i < nu; ++i) x[i] = y[i] / lam;
    }
    free(x); free(y); free(tu); free(tg); free(tp);
    return sqrt(lam);
}

/* ------------------------------------------------------------------------- */
/* Chambolle-Pock for dynamic tomography (Sec. 3, Fig. 2), on the            */
/* coefficients u (f = PhiF u on the frame grid, R_alpha = R):               */
/*   h1 <- (h1 + sigma R ut - sigma g) / (1 + sigma)                         */
/*   h2 <- project(h2 + sigma D ut, lambda1)        pointwise                */
/*   u  <- u - tau R* h1 - tau D^T h2               (D^T = -PhiF^T div)      */
/*   ut <- u + theta (u - u_old)                                             */
/* h1 = h2 = 0 and ut = u at the start; tau = sigma = 0.99 / L with L the    */
/* operator norm above (tau sigma L^2 < 1).                                  */
/* ------------------------------------------------------------------------- */
int or_chambolle_pock(const or_problem *P, const double *g, double *u, int iters, double lambda1,
                      double lambda2, double theta_cp, double L, double *objective)
{
    i64 nu = nu_of(P), ng = ng_of(P), np = np_of(P);
    double *h1 = (double *)calloc((size_t)ng, sizeof(double));
    double *h2 = (double *)calloc((size_t)np, sizeof(double));
    double *ut = (double *)malloc(sizeof(double) * nu);
    double *uold = (double *)malloc(sizeof(double) * nu);
    double *tg = (double *)malloc(sizeof(double) * ng);
    double *tp = (double *)malloc(sizeof(double) * np);
    double *ta = (double *)malloc(sizeof(double) * nu);
    double *tb = (double *)malloc(sizeof(double) * nu);
    if (!h1 || !h2 || !ut || !uold || !tg || !tp || !ta || !tb) return -2;
    double sigma = 0.99 / L, tau = 0.99 / L;
    memcpy(ut, u, sizeof(double) * nu);
    for (int it = 0; it < iters; ++it) {
        or_dyn_fwd(ut, P->nx, P->ny, P->nz, P->m, P->K, P->theta, P->Phi, P->ns, tg);
        for (i64 i = 0; i < ng; ++i) h1[i] = (h1[i] + sigma * tg[i] - sigma * g[i]) / (1.0 + sigma);
        or_D(ut, P->nx, P->ny, P->nz, P->m, P->PhiF, P->nt, lambda2, tp);
        for (i64 q = 0; q < np / 4; ++q) {
            double h[4];
            for (int c = 0; c < 4; ++c) h[c] = h2[q * 4 + c] + sigma * tp[q * 4 + c];
            or_project4(h, lambda1, h2 + q * 4);
        }
        or_dyn_adj(h1, P->nx, P->ny, P->nz, P->m, P->K, P->theta, P->Phi, P->ns, ta);
        or_DT(h2, P->nx, P->ny, P->nz, P->m, P->PhiF, P->nt, lambda2, tb);
        memcpy(uold, u, sizeof(double) * nu);
        for (i64 i = 0; i < nu; ++i) u[i] = u[i] - tau * ta[i] - tau * tb[i];
        for (i64 i = 0; i < nu; ++i) ut[i] = u[i] + theta_cp * (u[i] - uold[i]);
        if (objective) objective[it] = or_objective(P, g, u, lambda1, lambda2);
    }
    free(h1); free(h2); free(ut); free(uold); free(tg); free(tp); free(ta); free(tb);
    return 0;
}

/* Flat-argument entry points for the ctypes wrapper. */
static or_problem mk(int nx, int ny, int nz, int ns, int K, int m, int nt, const double *theta,
                     const double *Phi, const double *PhiF)
{
    or_problem P = {nx, ny, nz, ns, K, m, nt, theta, Phi, PhiF};
    return P;
}

int or_admm_cg_flat(int nx, int ny, int nz, int ns, int K, int m, int nt, const double *theta,
                    const double *Phi, const double *PhiF, const double *g, double *u, int iters,
                    int n_cg, double lambda1, double lambda2, double rho, double *objective,
                    double *primal_res)
{
    or_problem P = mk(nx, ny, nz, ns, K, m, nt, theta, Phi, PhiF);
    return or_admm_cg(&P, g, u, iters, n_cg, lambda1, lambda2, rho, objective, primal_res);
}

int or_chambolle_pock_flat(int nx, int ny, int nz, int ns, int K, int m, int nt,
                           const double *theta, const double *Phi, const double *PhiF,
                           const double *g, double *u, int iters, double lambda1, double lambda2,
                           double theta_cp, double L, double *objective)
{
    or_problem P = mk(nx, ny, nz, ns, K, m, nt, theta, Phi, PhiF);
    return or_chambolle_pock(&P, g, u, iters, lambda1, lambda2, theta_cp, L, objective);
}

double or_power_norm_flat(int nx, int ny, int nz, int ns, int K, int m, int nt,
                          const double *theta, const double *Phi, const double *PhiF,
                          double lambda2, int iters)
{
    or_problem P = mk(nx, ny, nz, ns, K, m, nt, theta, Phi, PhiF);
    return or_power_norm(&P, lambda2, iters);
}

double or_objective_flat(int nx, int ny, int nz, int ns, int K, int m, int nt,
                         const double *theta, const double *Phi, const double *PhiF,
                         const double *g, const double *u, double lambda1, double lambda2)
{
    or_problem P = mk(nx, ny, nz, ns, K, m, nt, theta, Phi, PhiF);
    return or_objective(&P, g, u, lambda1, lambda2);
}

/* ------------------------------------------------------------------------- */
/* FBP initial guess (Sec. 5: the iterations start from the filtered         */
/* back-projection reconstruction, with the Shepp-Logan filter).             */
/*                                                                           */
/* Filter: the discrete Shepp-Logan kernel at unit bin spacing,              */
/*     h(n) = -2 / (pi^2 (4 n^2 - 1)),                                       */
/* applied as a linear (zero-padded) convolution along s:                    */
/*     q[b] = sum_{b'} h(b - b') g[b'].                                      */
/* Its frequency response is |sin(w/2)| / pi, the ramp |w| / (2 pi) of the   */
/* continuous inversion formula rolled off towards the Nyquist frequency.    */
/* ------------------------------------------------------------------------- */
double or_shepp_logan_tap(i64 n)
{
    double nn = (double)n;
    return -2.0 / (M_PI * M_PI * (4.0 * nn * nn - 1.0));
}

void or_shepp_logan_filter(const double *g, i64 rows, int ns, double *q)
{
#pragma omp parallel for schedule(static)
    for (i64 r = 0; r < rows; ++r) {
        const double *gr = g + r * ns;
        double *qr = q + r * ns;
        for (int b = 0; b < ns; ++b) {
            double acc = 0.0;
            for (int bp = 0; bp < ns; ++bp) acc += or_shepp_logan_tap((i64)b - bp) * gr[bp];
            qr[b] = acc;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Windowed FBP images.  Projection k belongs to time window                 */
/*     w(k) = min(nw - 1, max(0, floor(t_k nw)))                             */
/* (one window per half-turn when nw is the number of half-turns, as the FBP */
/* frames of Sec. 5 are formed from the projections of one interval of       */
/* length pi).  With K_w projections in window w spread evenly over whole    */
/* half-turns, the angular integral over [0, pi) of the inversion formula is */
/* (pi / K_w) times the sum over the window, so                              */
/*     f[z][w] = (pi / K_w) sum_{k in w} R*_{theta_k} q[z][k]                */
/* with R* the exact Joseph transpose above; empty windows give 0.           */
/* f [nz][nw][ny][nx].                                                       */
/* ------------------------------------------------------------------------- */
int or_fbp_windows(const double *g, int nx, int ny, int nz, int K, const double *theta,
                   const double *t, int ns, int nw, double *f)
{
    i64 npix = (i64)nx * ny;
    double *q = (double *)malloc(sizeof(double) * (size_t)nz * K * ns);
    int *win = (int *)malloc(sizeof(int) * (size_t)K);
    i64 *cnt = (i64 *)calloc((size_t)nw, sizeof(i64));
    if (!q || !win || !cnt) return -2;
    or_shepp_logan_filter(g, (i64)nz * K, ns, q);
    for (int k = 0; k < K; ++k) {
        double x = floor(t[k] * nw);
        int w = x < 0.0 ? 0 : (x > nw - 1 ? nw - 1 : (int)x);
        win[k] = w;
        cnt[w] += 1;
    }
    memset(f, 0, sizeof(double) * (size_t)nz * nw * npix);
#pragma omp parallel for schedule(dynamic)
    for (int z = 0; z < nz; ++z) {
        double *tmp = (double *)malloc(sizeof(double) * npix);
        for (int k = 0; k < K; ++k) {
            or_joseph_adj_slice(q + ((i64)z * K + k) * ns, ns, theta[k], nx, ny, tmp);
            double *fw = f + ((i64)z * nw + win[k]) * npix;
            for (i64 p = 0; p < npix; ++p) fw[p] += tmp[p];
        }
        for (int w = 0; w < nw; ++w) {
            double sc = cnt[w] > 0 ? M_PI / (double)cnt[w] : 0.0;
            double *fw = f + ((i64)z * nw + w) * npix;
            for (i64 p = 0; p < npix; ++p) fw[p] *= sc;
        }
        free(tmp);
    }
    free(q); free(win); free(cnt);
    return 0;
}
