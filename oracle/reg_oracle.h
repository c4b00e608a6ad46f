/*
 * FP64 CPU oracle for matrix-free NGF + curvature registration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA path.
 *
 * Model: Budelmann, Koenig, Papenberg, Lellmann, "Fully-deformable 3D image
 * registration in two seconds" (BVM 2019), Sec. 2.1 (Eq. 1), Sec. 2.2
 * (Eq. 2 NGF, Eq. 3 node-centric P^T gather), with the discretisation choices
 * the paper leaves open fixed as listed beside each function.
 *
 * Conventions (all arrays are x-fastest: i = x + m_x (y + m_y z)):
 *   image grid m[3], spacing h[3] (mm); voxel centre x_{i,d} = (i_d + 1/2) h_d.
 *   deformation grid mn[3] nodes, nodal on the same box [0, m_d h_d]:
 *   node k at xi_{k,d} = k_d H_d, H_d = m_d h_d / (mn_d - 1).
 *   u is the displacement at the nodes, 3 planes of mn[0]*mn[1]*mn[2] values
 *   (component c at u[c*nn + k]); the deformation is y = xi + u.
 */
#ifndef REG_ORACLE_H
#define REG_ORACLE_H
#include <stddef.h>
#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_LEVELS 8
#define ORC_MAX_MEM 16

/* node spacing H_d = m_d h_d / (mn_d - 1) of the deformation grid (Sec. 2.1;
 * reading R1) */
void orc_node_spacing(const int m[3], const double h[3], const int mn[3], double H[3]);

/* grid conversion P (Sec. 2.1, Eq. 1): yhat_i = sum_k prod_d phi(x_{i,d}/H_d - k_d) u_k,
 * phi the 1D hat function; one component, u has mn[0]*mn[1]*mn[2] values */
void orc_P(const int m[3], const double h[3], const int mn[3], const double *u, double *yhat);

/* its transpose as the conflict-free node-centric gather of Eq. 3 (Sec. 2.2):
 * out_k = sum_{i in Omega_1 x Omega_2 x Omega_3} omega * r_i */
void orc_PT(const int m[3], const double h[3], const int mn[3], const double *r, double *out);

/* per-dimension index set Omega_d(k) and weights omega of Eq. 3 for one node
 * index k of one dimension: writes first voxel index and up to max_w weights,
 * returns the count */
int orc_PT_table(int m, double h, int mn, int k, int *first, double *w, int max_w);

/* trilinear interpolation of T at n physical points p (3 planes of n) as used
 * for T(P y) in Eq. 1 (Sec. 2.1), zero extension outside the image (reading
 * R5); value and interpolant gradient */
void orc_interp(const int m[3], const double h[3], const double *T, size_t n,
                const double *p, double *val, double *grad /* 3 planes of n */);

/* NGF distance (Eq. 2) of the deformed template Tw against R over interior
 * voxels; writes v = d psi_i / d (grad Tw_i) (3 planes) and returns D */
double orc_ngf(const int m[3], const double h[3], const double *Tw, const double *R,
               double tau, double rho, double *v);

/* adjoint of the central-difference gradient applied to v, times hbar/2: the
 * chain-rule step of Sec. 2.2 "Distance measure and gradient computation" */
void orc_ngf_adjoint(const int m[3], const double h[3], const double *v, double *g);

/* curvature regulariser (Sec. 2.1; Fischer-Modersitzki): S and grad S for the
 * 3 components of u; returns S */
double orc_curvature(const int mn[3], const double H[3], const double *u, double *gradS);

/* full objective J = D + alpha S (Eq. 1) and its gradient w.r.t. u (3 planes),
 * in the steps of Sec. 2.2 "Evaluating the objective function" */
void orc_objective(const int m[3], const double h[3], const double *R, const double *T,
                   const int mn[3], const double *u, double tau, double rho, double alpha,
                   double *J, double *D, double *S, double *grad);

/* pyramid (Sec. 2.2 "Generating the multi-level pyramid"; reading R4): one
 * 2x2x2 mean step; out dims ceil(m/2); an odd dimension replicates its last slab */
void orc_restrict(const int m[3], const double *img, double *out);

/* nodal trilinear prolongation of a displacement (3 planes) between two nodal
 * grids spanning the boxes ext_c and ext_f (mm): the coarse-to-fine step of the
 * multi-level scheme (Sec. 2.1) */
void orc_prolong(const int mn_c[3], const double ext_c[3], const double *uc,
                 const int mn_f[3], const double ext_f[3], double *uf);

/* L-BFGS two-loop recursion (Nocedal 1980): r = H g for pairs s_j, y_j
 * (count pairs, oldest first, each n values) with H0 = gamma I */
void orc_two_loop(size_t n, int count, const double *S, const double *Y,
                  const double *g, double gamma, double *r);

typedef struct {
    double tau, rho, alpha;
    double c1;                 /* Armijo constant */
    double tol_grad_rel;       /* stop when ||g|| <= tol * ||g0|| */
    double tol_j_rel;          /* stop when |J_{k-1}-J_k| <= tol (1+|J0|) ... */
    int tol_j_count;           /* ... for this many consecutive iterations */
    int levels;                /* pyramid levels, level 0 = finest */
    int mem;                   /* L-BFGS memory */
    int max_backtracks;        /* Armijo trials per line search */
    int fixed_iters;           /* 1: only the iteration cap stops a level */
    int start_level;           /* coarsest level solved; -1 = levels-1 */
    int max_iter[ORC_MAX_LEVELS];
    int node_dims[ORC_MAX_LEVELS][3]; /* 0 = rule m_d/2 + 1 */
} orc_config;

typedef struct {
    int iters[ORC_MAX_LEVELS];
    int evals[ORC_MAX_LEVELS];
    int status[ORC_MAX_LEVELS];  /* 0 ok, 1 line search failed */
    double J[ORC_MAX_LEVELS];
    double D[ORC_MAX_LEVELS];
    double S[ORC_MAX_LEVELS];
    int mn[ORC_MAX_LEVELS][3];
    int m[ORC_MAX_LEVELS][3];
} orc_stats;

/* level-wise node dims and image dims of a pyramid (readings R1, R4) */
void orc_level_dims(const int m[3], const orc_config *cfg, int level, int m_out[3], int mn_out[3]);

/* multilevel L-BFGS registration (Sec. 2.1; readings R9, R10); u_init on the
 * start level's node grid (NULL = zero); u_out on the finest node grid;
 * returns 0 or 1 (a level ended on a failed line search) */
int orc_register(const int m[3], const double h[3], const double *R, const double *T,
                 const orc_config *cfg, const double *u_init, double *u_out, orc_stats *st);

/* objective callback of the L-BFGS driver: returns J(u) and writes its
 * gradient g (n values) */
typedef double (*orc_eval_fn)(void *ctx, const double *u, double *g);

/* L-BFGS with Armijo backtracking on any objective (Sec. 2.1 "L-BFGS", Nocedal
 * 1980; readings R9, R10): memory cfg->mem, first step -g Hmin / ||g||_inf,
 * curvature-pair test, reset and one p0 retry on a failed search, and the
 * stopping tests of cfg; u in/out (n values); returns 0, or 1 when a line
 * search failed twice.  evals counts calls of fn. */
int orc_lbfgs(size_t n, orc_eval_fn fn, void *ctx, double Hmin, const orc_config *cfg, int max_iter,
              double *u, int *iters, int *evals, double *J_out);

/* one L-BFGS level on fixed images (Sec. 2.1; readings R9, R10; exposed for
 * tests); u in/out */
int orc_lbfgs_level(const int m[3], const double h[3], const double *R, const double *T,
                    const int mn[3], const orc_config *cfg, int max_iter, double *u,
                    int *iters, int *evals, double *J_out);

int orc_num_threads(void);

/* 1: every reduction (D, S, dot products, norms) uses compensated summation in
 * index order; 0 (default): the plain running sum in index order. */
void orc_set_compensated_sums(int on);
/* that reduction of a[0 .. n-1] */
double orc_sum(size_t n, const double *a);

#ifdef __cplusplus
}
#endif
#endif
