/*
 * FP64 CPU oracle for matrix-free NGF + curvature registration.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg.  Shares no code with the CUDA path.
 *
 * Every step is written the plain way: intermediates (yhat, deformed template,
 * its interpolant gradient, v, g, r) are materialised as full arrays, loops run
 * in index order, and sums are taken sequentially in index order after a
 * parallel map.  OpenMP only splits independent per-voxel / per-node maps.
 *
 * Readings of places the paper leaves open (same numbering in the design notes):
 *  R1 image grid cell-centred, deformation grid nodal on the same box,
 *     H_d = m_d h_d / (mn_d - 1); the default node count is m_d/2 + 1.
 *  R2 the unknown is the displacement u, y = xi + u.
 *  R3 P^T is applied to the gradient only.
 *  R4 pyramid = 2x2x2 mean, spacing doubles, odd dims replicate the last slab.
 *  R5 template interpolation is trilinear with zero extension; its gradient
 *     uses the floor cell.
 *  R6 curvature: 7-point Laplacian on interior nodes only.
 *  R7 tau and rho are separate parameters (the workloads set tau = rho = eta).
 *  R8 NGF sums over interior voxels, central differences there.
 *  R9 L-BFGS (two-loop, H0 = gamma I with gamma = s'y / y'y of the newest pair,
 *     first step p0 = -g min_d H_d / ||g||_inf, curvature test
 *     s'y > 1e-10 ||s|| ||y||, reset on ascent direction, Armijo backtracking
 *     t = 1, 1/2, ... with one p0 retry after a failed search).
 *  R10 stopping: iteration cap, ||g|| <= tol ||g0||, or tol_j_count consecutive
 *     |J_{k-1} - J_k| <= tol_j (1 + |J0|).
 */
#include "reg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX3(x, y, z, nx, ny) ((size_t)(x) + (size_t)(nx) * ((size_t)(y) + (size_t)(ny) * (size_t)(z)))

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* 1D hat (linear B-spline) basis function */
static double hat(double t)
{
    double a = fabs(t);
    return a < 1.0 ? 1.0 - a : 0.0;
}

static size_t vol(const int m[3]) { return (size_t)m[0] * (size_t)m[1] * (size_t)m[2]; }

/* Every reduction of the oracle (D, S, the L-BFGS dot products and norms) adds
 * its terms one by one in index order.  With compensated sums switched on it
 * carries the rounding error of each addition in a second word (Neumaier's
 * variant of Kahan summation, 1974), so the result is the exact sum up to
 * about one rounding; with them off (the default) it is the plain running
 * sum. */
static int g_compensated = 0;

void orc_set_compensated_sums(int on) { g_compensated = on != 0; }

typedef struct {
    double s, c;
} acc_t;

static void acc_add(acc_t *a, double x)
{
    if (!g_compensated) {
        a->s += x;
        return;
    }
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

static double acc_value(const acc_t *a) { return g_compensated ? a->s + a->c : a->s; }

/* the reduction above applied to a[0 .. n-1] (exported to pin it) */
double orc_sum(size_t n, const double *a)
{
    acc_t s = {0.0, 0.0};
    for (size_t i = 0; i < n; i++)
        acc_add(&s, a[i]);
    return acc_value(&s);
}

void orc_node_spacing(const int m[3], const double h[3], const int mn[3], double H[3])
{
    for (int d = 0; d < 3; d++)
        H[d] = (double)m[d] * h[d] / (double)(mn[d] - 1);
}

/* ---------------------------------------------------------------------------
 * Grid conversion P (Sec. 2.1, Eq. 1; Sec. 2.2 "Grid conversion"):
 *   yhat_i = sum_k  prod_d phi(x_{i,d} / H_d - k_d)  u_k,
 * the sum running over the nodes whose hat functions are non-zero at x_i.
 * ------------------------------------------------------------------------- */
void orc_P(const int m[3], const double h[3], const int mn[3], const double *u, double *yhat)
{
    double H[3];
    orc_node_spacing(m, h, mn, H);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < m[2]; z++)
        for (int y = 0; y < m[1]; y++)
            for (int x = 0; x < m[0]; x++) {
                int i[3] = {x, y, z};
                double t[3];
                int k0[3];
                for (int d = 0; d < 3; d++) {
                    t[d] = (i[d] + 0.5) * h[d] / H[d];
                    k0[d] = (int)floor(t[d]);
                }
                double s = 0.0;
                for (int c = 0; c < 8; c++) {
                    int k[3] = {k0[0] + (c & 1), k0[1] + ((c >> 1) & 1), k0[2] + ((c >> 2) & 1)};
                    if (k[0] < 0 || k[1] < 0 || k[2] < 0 || k[0] >= mn[0] || k[1] >= mn[1] || k[2] >= mn[2])
                        continue;
                    double w = hat(t[0] - k[0]) * hat(t[1] - k[1]) * hat(t[2] - k[2]);
                    s += w * u[IDX3(k[0], k[1], k[2], mn[0], mn[1])];
                }
                yhat[IDX3(x, y, z, m[0], m[1])] = s;
            }
}

/* ---------------------------------------------------------------------------
 * P^T as the node-centric gather of Eq. 3 (Sec. 2.2): node k sums
 * omega * r_i over i in Omega_1(k_1) x Omega_2(k_2) x Omega_3(k_3); the index
 * sets and the 1D weights are determined beforehand, one dimension at a time.
 * ------------------------------------------------------------------------- */
int orc_PT_table(int m, double h, int mn, int k, int *first, double *w, int max_w)
{
    double H = (double)m * h / (double)(mn - 1);
    int cnt = 0;
    *first = -1;
    for (int i = 0; i < m; i++) {
        double om = hat((i + 0.5) * h / H - k);
        if (om > 0.0) {
            if (cnt == 0)
                *first = i;
            if (cnt < max_w)
                w[cnt] = om;
            cnt++;
        }
    }
    return cnt;
}

typedef struct {
    int *first, *cnt;
    double *w; /* [k * maxw + j] */
    int maxw;
} pt_table;

static void pt_table_build(int m, double h, int mn, pt_table *t)
{
    double ratio = (double)m / (double)(mn - 1);
    t->maxw = (int)ceil(2.0 * ratio) + 2;
    t->first = (int *)malloc(sizeof(int) * mn);
    t->cnt = (int *)malloc(sizeof(int) * mn);
    t->w = (double *)calloc((size_t)mn * t->maxw, sizeof(double));
    for (int k = 0; k < mn; k++)
        t->cnt[k] = orc_PT_table(m, h, mn, k, &t->first[k], t->w + (size_t)k * t->maxw, t->maxw);
}

static void pt_table_free(pt_table *t)
{
    free(t->first);
    free(t->cnt);
    free(t->w);
}

void orc_PT(const int m[3], const double h[3], const int mn[3], const double *r, double *out)
{
    pt_table tab[3];
    for (int d = 0; d < 3; d++)
        pt_table_build(m[d], h[d], mn[d], &tab[d]);
#pragma omp parallel for schedule(static)
    for (int kz = 0; kz < mn[2]; kz++)
        for (int ky = 0; ky < mn[1]; ky++)
            for (int kx = 0; kx < mn[0]; kx++) {
                const double *wx = tab[0].w + (size_t)kx * tab[0].maxw;
                const double *wy = tab[1].w + (size_t)ky * tab[1].maxw;
                const double *wz = tab[2].w + (size_t)kz * tab[2].maxw;
                double s = 0.0;
                for (int c = 0; c < tab[2].cnt[kz]; c++)
                    for (int b = 0; b < tab[1].cnt[ky]; b++)
                        for (int a = 0; a < tab[0].cnt[kx]; a++) {
                            int ix = tab[0].first[kx] + a, iy = tab[1].first[ky] + b, iz = tab[2].first[kz] + c;
                            s += wx[a] * wy[b] * wz[c] * r[IDX3(ix, iy, iz, m[0], m[1])];
                        }
                out[IDX3(kx, ky, kz, mn[0], mn[1])] = s;
            }
    for (int d = 0; d < 3; d++)
        pt_table_free(&tab[d]);
}

/* ---------------------------------------------------------------------------
 * Template interpolation T(p) (Sec. 2.1, "interpolate the deformed template"):
 * T(p) = sum_j T_j prod_d phi(p_d / h_d - 1/2 - j_d), T_j = 0 outside the image
 * (R5).  The gradient is that of the interpolant inside the cell
 * c = floor(p/h - 1/2).
 * ------------------------------------------------------------------------- */
static void interp_voxel_units(const int m[3], const double h[3], const double *T, const double t[3],
                               double *val, double grad[3])
{
    double f[3];
    long c[3];
    for (int d = 0; d < 3; d++) {
        c[d] = (long)floor(t[d]);
        f[d] = t[d] - (double)c[d];
    }
    double v = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    for (int cz = 0; cz < 2; cz++)
        for (int cy = 0; cy < 2; cy++)
            for (int cx = 0; cx < 2; cx++) {
                long jx = c[0] + cx, jy = c[1] + cy, jz = c[2] + cz;
                double Tj = 0.0;
                if (jx >= 0 && jy >= 0 && jz >= 0 && jx < m[0] && jy < m[1] && jz < m[2])
                    Tj = T[IDX3(jx, jy, jz, m[0], m[1])];
                double wx = cx ? f[0] : 1.0 - f[0];
                double wy = cy ? f[1] : 1.0 - f[1];
                double wz = cz ? f[2] : 1.0 - f[2];
                double dx = (cx ? 1.0 : -1.0) / h[0];
                double dy = (cy ? 1.0 : -1.0) / h[1];
                double dz = (cz ? 1.0 : -1.0) / h[2];
                v += wx * wy * wz * Tj;
                g0 += dx * wy * wz * Tj;
                g1 += wx * dy * wz * Tj;
                g2 += wx * wy * dz * Tj;
            }
    *val = v;
    grad[0] = g0;
    grad[1] = g1;
    grad[2] = g2;
}

/* T and its gradient at a physical point p (mm): t = p / h - 1/2 in voxel units. */
static void interp_point(const int m[3], const double h[3], const double *T, const double p[3],
                         double *val, double grad[3])
{
    double t[3];
    for (int d = 0; d < 3; d++)
        t[d] = p[d] / h[d] - 0.5;
    interp_voxel_units(m, h, T, t, val, grad);
}

void orc_interp(const int m[3], const double h[3], const double *T, size_t n, const double *p,
                double *val, double *grad)
{
#pragma omp parallel for schedule(static)
    for (long q = 0; q < (long)n; q++) {
        double pt[3] = {p[q], p[n + q], p[2 * n + q]}, g[3];
        interp_point(m, h, T, pt, &val[q], g);
        if (grad) {
            grad[q] = g[0];
            grad[n + q] = g[1];
            grad[2 * n + q] = g[2];
        }
    }
}

/* ---------------------------------------------------------------------------
 * NGF distance, Eq. 2 (Sec. 2.2 "Distance measure and gradient computation"):
 *   D = hbar/2 sum_i (1 - c_i^2),
 *   c_i = (<a, b> + tau rho) / (||a||_tau ||b||_rho),  ||z||_e = sqrt(<z,z> + e^2),
 * a = grad of the deformed template, b = grad R, central differences on the
 * interior voxels (R8).  Also v_i = d(1 - c_i^2)/d a:
 *   v = -2 c (b / (||a|| ||b||) - c a / ||a||^2).
 * ------------------------------------------------------------------------- */
double orc_ngf(const int m[3], const double h[3], const double *Tw, const double *R, double tau,
               double rho, double *v)
{
    size_t nv = vol(m);
    size_t st[3] = {1, (size_t)m[0], (size_t)m[0] * m[1]};
    double *psi = (double *)calloc(nv, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int z = 0; z < m[2]; z++)
        for (int y = 0; y < m[1]; y++)
            for (int x = 0; x < m[0]; x++) {
                size_t i = IDX3(x, y, z, m[0], m[1]);
                v[i] = v[nv + i] = v[2 * nv + i] = 0.0;
                int interior = x >= 1 && y >= 1 && z >= 1 && x <= m[0] - 2 && y <= m[1] - 2 && z <= m[2] - 2;
                if (!interior)
                    continue;
                double a[3], b[3];
                for (int d = 0; d < 3; d++) {
                    a[d] = (Tw[i + st[d]] - Tw[i - st[d]]) / (2.0 * h[d]);
                    b[d] = (R[i + st[d]] - R[i - st[d]]) / (2.0 * h[d]);
                }
                double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
                double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
                double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
                double na = sqrt(aa + tau * tau), nb = sqrt(bb + rho * rho);
                double c = (ab + tau * rho) / (na * nb);
                psi[i] = 1.0 - c * c;
                for (int d = 0; d < 3; d++)
                    v[d * nv + i] = -2.0 * c * (b[d] / (na * nb) - c * a[d] / (na * na));
            }
    acc_t D = {0.0, 0.0};
    for (size_t i = 0; i < nv; i++)
        acc_add(&D, psi[i]);
    free(psi);
    return 0.5 * h[0] * h[1] * h[2] * acc_value(&D);
}

/* g_j = d D / d Tw_j = hbar/2 sum_d (v_d[j - e_d] - v_d[j + e_d]) / (2 h_d),
 * the chain rule through the central differences (Sec. 2.2, matrix-free
 * gradient); v is zero outside the volume. */
void orc_ngf_adjoint(const int m[3], const double h[3], const double *v, double *g)
{
    size_t nv = vol(m);
    double hbar = h[0] * h[1] * h[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < m[2]; z++)
        for (int y = 0; y < m[1]; y++)
            for (int x = 0; x < m[0]; x++) {
                int j[3] = {x, y, z};
                double s = 0.0;
                for (int d = 0; d < 3; d++) {
                    int lo[3] = {x, y, z}, hi[3] = {x, y, z};
                    lo[d] -= 1;
                    hi[d] += 1;
                    double vlo = 0.0, vhi = 0.0;
                    if (j[d] - 1 >= 0)
                        vlo = v[d * nv + IDX3(lo[0], lo[1], lo[2], m[0], m[1])];
                    if (j[d] + 1 < m[d])
                        vhi = v[d * nv + IDX3(hi[0], hi[1], hi[2], m[0], m[1])];
                    s += (vlo - vhi) / (2.0 * h[d]);
                }
                g[IDX3(x, y, z, m[0], m[1])] = 0.5 * hbar * s;
            }
}

/* ---------------------------------------------------------------------------
 * Curvature regulariser (Sec. 2.1; penalises (Laplace y_c)^2):
 *   w_c = L u_c on interior nodes (7-point stencil, spacing H), 0 elsewhere (R6)
 *   S = hbar_y / 2 sum_c sum_k w_c[k]^2,   grad_c S = hbar_y L^T w_c.
 * ------------------------------------------------------------------------- */
double orc_curvature(const int mn[3], const double H[3], const double *u, double *gradS)
{
    size_t nn = vol(mn);
    size_t st[3] = {1, (size_t)mn[0], (size_t)mn[0] * mn[1]};
    double hy = H[0] * H[1] * H[2];
    double iH2[3] = {1.0 / (H[0] * H[0]), 1.0 / (H[1] * H[1]), 1.0 / (H[2] * H[2])};
    double *w = (double *)malloc(sizeof(double) * nn);
    acc_t S = {0.0, 0.0};
    for (int c = 0; c < 3; c++) {
        const double *uc = u + c * nn;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < mn[2]; z++)
            for (int y = 0; y < mn[1]; y++)
                for (int x = 0; x < mn[0]; x++) {
                    size_t k = IDX3(x, y, z, mn[0], mn[1]);
                    int interior = x >= 1 && y >= 1 && z >= 1 && x <= mn[0] - 2 && y <= mn[1] - 2 && z <= mn[2] - 2;
                    double lap = 0.0;
                    if (interior)
                        for (int d = 0; d < 3; d++)
                            lap += (uc[k + st[d]] - 2.0 * uc[k] + uc[k - st[d]]) * iH2[d];
                    w[k] = lap;
                }
        for (size_t k = 0; k < nn; k++)
            acc_add(&S, w[k] * w[k]);
        if (gradS) {
            double *gc = gradS + c * nn;
#pragma omp parallel for schedule(static)
            for (int z = 0; z < mn[2]; z++)
                for (int y = 0; y < mn[1]; y++)
                    for (int x = 0; x < mn[0]; x++) {
                        int j[3] = {x, y, z};
                        size_t k = IDX3(x, y, z, mn[0], mn[1]);
                        double s = 0.0;
                        for (int d = 0; d < 3; d++) {
                            double wl = j[d] - 1 >= 0 ? w[k - st[d]] : 0.0;
                            double wh = j[d] + 1 < mn[d] ? w[k + st[d]] : 0.0;
                            s += (wl + wh - 2.0 * w[k]) * iH2[d];
                        }
                        gc[k] = hy * s;
                    }
        }
    }
    free(w);
    return 0.5 * hy * acc_value(&S);
}

/* ---------------------------------------------------------------------------
 * Objective J = D(R, T(P y)) + alpha S(y) and grad_u J (Eq. 1), in the three
 * steps of Sec. 2.2 "Evaluating the objective function":
 *   (1) yhat = P u;  (2) D and its gradient on the image grid;  (3) P^T.
 * ------------------------------------------------------------------------- */
void orc_objective(const int m[3], const double h[3], const double *R, const double *T, const int mn[3],
                   const double *u, double tau, double rho, double alpha, double *J, double *D, double *S,
                   double *grad)
{
    size_t nv = vol(m), nn = vol(mn);
    double H[3];
    orc_node_spacing(m, h, mn, H);
    double *yhat = (double *)malloc(sizeof(double) * 3 * nv);
    double *Tw = (double *)malloc(sizeof(double) * nv);
    double *dT = (double *)malloc(sizeof(double) * 3 * nv);
    double *v = (double *)malloc(sizeof(double) * 3 * nv);
    double *g = (double *)malloc(sizeof(double) * nv);

    /* (1) grid conversion, per component */
    for (int c = 0; c < 3; c++)
        orc_P(m, h, mn, u + c * nn, yhat + c * nv);
    /* (2) deformed template at p_i = x_i + yhat_i (P reproduces the node
     * positions xi) and its interpolant gradient.  With x_i = (i + 1/2) h (R1)
     * the voxel coordinate p_i / h - 1/2 is exactly i + yhat_i / h; it is formed
     * that way, so that a sample on a cell face (yhat a whole number of voxels)
     * lands on the integer and takes the cell to its right (R5), instead of
     * rounding below it through the product (i + 1/2) h. */
#pragma omp parallel for schedule(static)
    for (int z = 0; z < m[2]; z++)
        for (int y = 0; y < m[1]; y++)
            for (int x = 0; x < m[0]; x++) {
                size_t i = IDX3(x, y, z, m[0], m[1]);
                double t[3] = {x + yhat[i] / h[0], y + yhat[nv + i] / h[1], z + yhat[2 * nv + i] / h[2]};
                double gr[3];
                interp_voxel_units(m, h, T, t, &Tw[i], gr);
                dT[i] = gr[0];
                dT[nv + i] = gr[1];
                dT[2 * nv + i] = gr[2];
            }
    /* NGF, chain rule */
    double Dv = orc_ngf(m, h, Tw, R, tau, rho, v);
    orc_ngf_adjoint(m, h, v, g);
    double *r = yhat; /* reuse: r_c = g * dT_c */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)nv; i++)
        for (int c = 0; c < 3; c++)
            r[c * nv + i] = g[i] * dT[c * nv + i];
    /* (3) back to the deformation grid */
    for (int c = 0; c < 3; c++)
        orc_PT(m, h, mn, r + c * nv, grad + c * nn);

    double *gS = (double *)malloc(sizeof(double) * 3 * nn);
    double Sv = orc_curvature(mn, H, u, gS);
    for (size_t k = 0; k < 3 * nn; k++)
        grad[k] += alpha * gS[k];
    *D = Dv;
    *S = Sv;
    *J = Dv + alpha * Sv;
    free(gS);
    free(yhat);
    free(Tw);
    free(dT);
    free(v);
    free(g);
}

/* ---------------------------------------------------------------------------
 * Pyramid (Sec. 2.2 "Generating the multi-level pyramid"), reading R4.
 * ------------------------------------------------------------------------- */
void orc_restrict(const int m[3], const double *img, double *out)
{
    int mo[3] = {(m[0] + 1) / 2, (m[1] + 1) / 2, (m[2] + 1) / 2};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < mo[2]; z++)
        for (int y = 0; y < mo[1]; y++)
            for (int x = 0; x < mo[0]; x++) {
                double s = 0.0;
                for (int c = 0; c < 2; c++)
                    for (int b = 0; b < 2; b++)
                        for (int a = 0; a < 2; a++) {
                            int ix = 2 * x + a, iy = 2 * y + b, iz = 2 * z + c;
                            if (ix > m[0] - 1) ix = m[0] - 1;
                            if (iy > m[1] - 1) iy = m[1] - 1;
                            if (iz > m[2] - 1) iz = m[2] - 1;
                            s += img[IDX3(ix, iy, iz, m[0], m[1])];
                        }
                out[IDX3(x, y, z, mo[0], mo[1])] = s / 8.0;
            }
}

/* nodal trilinear prolongation (Sec. 2.1, multilevel): fine node j at j H_f is
 * evaluated with the coarse hat basis at t = j H_f / H_c */
void orc_prolong(const int mn_c[3], const double ext_c[3], const double *uc, const int mn_f[3],
                 const double ext_f[3], double *uf)
{
    size_t nc = vol(mn_c), nf = vol(mn_f);
    double Hc[3], Hf[3];
    for (int d = 0; d < 3; d++) {
        Hc[d] = ext_c[d] / (mn_c[d] - 1);
        Hf[d] = ext_f[d] / (mn_f[d] - 1);
    }
    for (int comp = 0; comp < 3; comp++) {
        const double *src = uc + comp * nc;
        double *dst = uf + comp * nf;
#pragma omp parallel for schedule(static)
        for (int z = 0; z < mn_f[2]; z++)
            for (int y = 0; y < mn_f[1]; y++)
                for (int x = 0; x < mn_f[0]; x++) {
                    int j[3] = {x, y, z};
                    double t[3];
                    int k0[3];
                    for (int d = 0; d < 3; d++) {
                        t[d] = j[d] * Hf[d] / Hc[d];
                        if (t[d] > mn_c[d] - 1)
                            t[d] = mn_c[d] - 1;
                        k0[d] = (int)floor(t[d]);
                        if (k0[d] > mn_c[d] - 2)
                            k0[d] = mn_c[d] - 2;
                    }
                    double s = 0.0;
                    for (int c = 0; c < 8; c++) {
                        int k[3] = {k0[0] + (c & 1), k0[1] + ((c >> 1) & 1), k0[2] + ((c >> 2) & 1)};
                        double w = hat(t[0] - k[0]) * hat(t[1] - k[1]) * hat(t[2] - k[2]);
                        s += w * src[IDX3(k[0], k[1], k[2], mn_c[0], mn_c[1])];
                    }
                    dst[IDX3(x, y, z, mn_f[0], mn_f[1])] = s;
                }
    }
}

/* ---------------------------------------------------------------------------
 * L-BFGS (Sec. 2.1; Nocedal 1980), reading R9.
 * ------------------------------------------------------------------------- */
static double dot(size_t n, const double *a, const double *b)
{
    acc_t s = {0.0, 0.0};
    for (size_t i = 0; i < n; i++)
        acc_add(&s, a[i] * b[i]);
    return acc_value(&s);
}

void orc_two_loop(size_t n, int count, const double *S, const double *Y, const double *g, double gamma,
                  double *r)
{
    double alpha[ORC_MAX_MEM], rho[ORC_MAX_MEM];
    double *q = r;
    memcpy(q, g, sizeof(double) * n);
    for (int j = count - 1; j >= 0; j--) {
        const double *s = S + (size_t)j * n, *y = Y + (size_t)j * n;
        rho[j] = 1.0 / dot(n, s, y);
        alpha[j] = rho[j] * dot(n, s, q);
        for (size_t i = 0; i < n; i++)
            q[i] -= alpha[j] * y[i];
    }
    for (size_t i = 0; i < n; i++)
        q[i] *= gamma;
    for (int j = 0; j < count; j++) {
        const double *s = S + (size_t)j * n, *y = Y + (size_t)j * n;
        double beta = rho[j] * dot(n, y, q);
        for (size_t i = 0; i < n; i++)
            q[i] += s[i] * (alpha[j] - beta);
    }
}

typedef struct {
    const int *m, *mn;
    const double *h, *R, *T;
    const orc_config *cfg;
} level_ctx;

/* the objective of one pyramid level (Eq. 1) as an L-BFGS callback */
static double level_eval(void *ctx, const double *u, double *g)
{
    const level_ctx *L = (const level_ctx *)ctx;
    double J, D, S;
    orc_objective(L->m, L->h, L->R, L->T, L->mn, u, L->cfg->tau, L->cfg->rho, L->cfg->alpha, &J, &D, &S, g);
    return J;
}

typedef struct {
    orc_eval_fn fn;
    void *ctx;
    int evals;
} counted_fn;

static double eval_counted(counted_fn *f, const double *u, double *g)
{
    f->evals++;
    return f->fn(f->ctx, u, g);
}

/* p0 = -g * Hmin / ||g||_inf: a first step of at most one node spacing (reading R9) */
static double first_direction(size_t n, const double *g, double Hmin, double *p)
{
    double gi = 0.0;
    for (size_t i = 0; i < n; i++)
        if (fabs(g[i]) > gi)
            gi = fabs(g[i]);
    double sc = gi > 0.0 ? Hmin / gi : 0.0;
    for (size_t i = 0; i < n; i++)
        p[i] = -sc * g[i];
    return dot(n, g, p);
}

/* Armijo backtracking: t = 1, 1/2, ...; accept J(u + t p) <= J + c1 t g'p (reading R9) */
static int line_search(counted_fn *f, const orc_config *cfg, size_t n, const double *u, const double *p,
                       double J, double gtp, double *ut, double *gt, double *Jt, double *t_out)
{
    double t = 1.0;
    for (int trial = 0; trial < cfg->max_backtracks; trial++) {
        for (size_t i = 0; i < n; i++)
            ut[i] = u[i] + t * p[i];
        *Jt = eval_counted(f, ut, gt);
        if (*Jt <= J + cfg->c1 * t * gtp) {
            *t_out = t;
            return 1;
        }
        t *= 0.5;
    }
    return 0;
}

int orc_lbfgs(size_t n, orc_eval_fn fn, void *ctx, double Hmin, const orc_config *cfg, int max_iter,
              double *u, int *iters, int *evals, double *J_out)
{
    int mem = cfg->mem < 1 ? 1 : (cfg->mem > ORC_MAX_MEM ? ORC_MAX_MEM : cfg->mem);
    counted_fn F = {fn, ctx, 0};

    double *g = (double *)malloc(sizeof(double) * n);
    double *gt = (double *)malloc(sizeof(double) * n);
    double *ut = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *Sm = (double *)malloc(sizeof(double) * n * mem);
    double *Ym = (double *)malloc(sizeof(double) * n * mem);
    double *tmp = (double *)malloc(sizeof(double) * n);
    int count = 0, status = 0, k = 0, small = 0;

    double Jt, t;
    double J = eval_counted(&F, u, g);
    double J0 = J, g0n = sqrt(dot(n, g, g));

    while (k < max_iter && g0n > 0.0) {
        int use_p0 = (count == 0);
        double gtp;
        if (use_p0) {
            gtp = first_direction(n, g, Hmin, p);
        } else {
            const double *sn = Sm + (size_t)(count - 1) * n, *yn = Ym + (size_t)(count - 1) * n;
            double gamma = dot(n, sn, yn) / dot(n, yn, yn);
            orc_two_loop(n, count, Sm, Ym, g, gamma, p);
            for (size_t i = 0; i < n; i++)
                p[i] = -p[i];
            gtp = dot(n, g, p);
            if (!(gtp < 0.0)) { /* not a descent direction: reset the memory */
                count = 0;
                use_p0 = 1;
                gtp = first_direction(n, g, Hmin, p);
            }
        }
        int ok = line_search(&F, cfg, n, u, p, J, gtp, ut, gt, &Jt, &t);
        if (!ok && !use_p0) { /* one retry from a fresh memory */
            count = 0;
            gtp = first_direction(n, g, Hmin, p);
            ok = line_search(&F, cfg, n, u, p, J, gtp, ut, gt, &Jt, &t);
        }
        if (!ok) {
            status = 1;
            break;
        }
        /* new pair s = t p, y = g_new - g, kept only if it passes the curvature test */
        double *snew = tmp, *ynew = ut;  /* ut is free again once copied to u below */
        memcpy(u, ut, sizeof(double) * n);
        for (size_t i = 0; i < n; i++) {
            snew[i] = t * p[i];
            ynew[i] = gt[i] - g[i];
        }
        double sy = dot(n, snew, ynew);
        double ss = dot(n, snew, snew), yy = dot(n, ynew, ynew);
        if (sy > 1e-10 * sqrt(ss) * sqrt(yy)) {
            if (count == mem) { /* drop the oldest pair */
                memmove(Sm, Sm + n, sizeof(double) * n * (mem - 1));
                memmove(Ym, Ym + n, sizeof(double) * n * (mem - 1));
                count--;
            }
            memcpy(Sm + (size_t)count * n, snew, sizeof(double) * n);
            memcpy(Ym + (size_t)count * n, ynew, sizeof(double) * n);
            count++;
        }
        double Jprev = J;
        memcpy(g, gt, sizeof(double) * n);
        J = Jt;
        k++;
        if (!cfg->fixed_iters) { /* reading R10 */
            if (sqrt(dot(n, g, g)) <= cfg->tol_grad_rel * g0n)
                break;
            if (fabs(Jprev - J) <= cfg->tol_j_rel * (1.0 + fabs(J0))) {
                if (++small >= cfg->tol_j_count)
                    break;
            } else {
                small = 0;
            }
        }
    }
    *iters = k;
    *evals = F.evals;
    *J_out = J;
    free(g);
    free(gt);
    free(ut);
    free(p);
    free(Sm);
    free(Ym);
    free(tmp);
    return status;
}

int orc_lbfgs_level(const int m[3], const double h[3], const double *R, const double *T, const int mn[3],
                    const orc_config *cfg, int max_iter, double *u, int *iters, int *evals, double *J_out)
{
    double H[3];
    orc_node_spacing(m, h, mn, H);
    level_ctx L = {m, mn, h, R, T, cfg};
    return orc_lbfgs(3 * vol(mn), level_eval, &L, fmin(H[0], fmin(H[1], H[2])), cfg, max_iter, u, iters, evals,
                     J_out);
}

void orc_level_dims(const int m[3], const orc_config *cfg, int level, int m_out[3], int mn_out[3])
{
    int ml[3] = {m[0], m[1], m[2]};
    for (int l = 0; l < level; l++)
        for (int d = 0; d < 3; d++)
            ml[d] = (ml[d] + 1) / 2;
    for (int d = 0; d < 3; d++) {
        m_out[d] = ml[d];
        int rule = ml[d] / 2 + 1;
        mn_out[d] = (cfg && cfg->node_dims[level][d] > 0) ? cfg->node_dims[level][d] : rule;
    }
}

int orc_register(const int m[3], const double h[3], const double *R, const double *T, const orc_config *cfg,
                 const double *u_init, double *u_out, orc_stats *st)
{
    int L = cfg->levels < 1 ? 1 : (cfg->levels > ORC_MAX_LEVELS ? ORC_MAX_LEVELS : cfg->levels);
    int start = cfg->start_level < 0 || cfg->start_level >= L ? L - 1 : cfg->start_level;
    double *Rl[ORC_MAX_LEVELS], *Tl[ORC_MAX_LEVELS];
    int ml[ORC_MAX_LEVELS][3], mnl[ORC_MAX_LEVELS][3];
    double hl[ORC_MAX_LEVELS][3];
    memset(st, 0, sizeof(*st));

    Rl[0] = (double *)R;
    Tl[0] = (double *)T;
    for (int l = 0; l < L; l++) {
        orc_level_dims(m, cfg, l, ml[l], mnl[l]);
        for (int d = 0; d < 3; d++) {
            hl[l][d] = h[d] * (double)(1 << l);
            st->m[l][d] = ml[l][d];
            st->mn[l][d] = mnl[l][d];
        }
        if (l > 0) {
            Rl[l] = (double *)malloc(sizeof(double) * vol(ml[l]));
            Tl[l] = (double *)malloc(sizeof(double) * vol(ml[l]));
            orc_restrict(ml[l - 1], Rl[l - 1], Rl[l]);
            orc_restrict(ml[l - 1], Tl[l - 1], Tl[l]);
        }
    }

    size_t n = 3 * vol(mnl[start]);
    double *u = (double *)calloc(n, sizeof(double));
    if (u_init)
        memcpy(u, u_init, sizeof(double) * n);
    int status = 0;
    for (int l = start; l >= 0; l--) {
        if (l < start) {
            double ext_c[3], ext_f[3];
            for (int d = 0; d < 3; d++) {
                ext_c[d] = ml[l + 1][d] * hl[l + 1][d];
                ext_f[d] = ml[l][d] * hl[l][d];
            }
            double *uf = (double *)malloc(sizeof(double) * 3 * vol(mnl[l]));
            orc_prolong(mnl[l + 1], ext_c, u, mnl[l], ext_f, uf);
            free(u);
            u = uf;
        }
        int it = 0, ev = 0;
        double J;
        int s = orc_lbfgs_level(ml[l], hl[l], Rl[l], Tl[l], mnl[l], cfg, cfg->max_iter[l], u, &it, &ev, &J);
        st->iters[l] = it;
        st->evals[l] = ev;
        st->status[l] = s;
        st->J[l] = J;
        if (s)
            status = 1;
    }
    memcpy(u_out, u, sizeof(double) * 3 * vol(mnl[0]));
    free(u);
    for (int l = 1; l < L; l++) {
        free(Rl[l]);
        free(Tl[l]);
    }
    return status;
}
